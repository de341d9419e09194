"""GB300 library for the real-space RPA correlation energy by Lanczos quadrature.

The compute path lives in ``csrc/`` (CUDA for sm_103a) behind the C ABI declared in
``include/rpa.h``; this module is the thin Python binding: it builds the shared library,
loads it, and marshals arguments for functions that carry the same names as the C entry
points.  Host arguments are numpy arrays; device arguments are CUDA tensors (torch), passed
by pointer.  Every call raises :class:`RpaError` on a non-OK status.  There is no fallback:
if the CUDA library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import glob
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "librpa.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
_LOCK = threading.Lock()
_LIB = None

# enums (include/rpa.h)
RPA_OK, RPA_EINVAL, RPA_ENOMEM, RPA_ECUDA, RPA_ENOCONV, RPA_EBREAKDOWN, RPA_ETIMEOUT, \
    RPA_ENOGAP, RPA_ESTATE = range(9)
RPA_HOST, RPA_DEVICE = 0, 1
RPA_PERIODIC, RPA_DIRICHLET = 0, 1
RPA_FP64, RPA_MIXED, RPA_MIXED_BF16 = 0, 1, 2
RPA_INTERP_NONE, RPA_INTERP_TRILINEAR, RPA_INTERP_TRICUBIC, RPA_INTERP_FOURIER = range(4)
RPA_F_LOG, RPA_F_X, RPA_F_X2 = range(3)
INTERP = {"none": 0, "linear": 1, "trilinear": 1, "cubic": 2, "tricubic": 2, "fourier": 3}


class RpaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


# -------------------------------------------------------------------------------------------
# build / load
# -------------------------------------------------------------------------------------------
def _sources():
    return sorted(glob.glob(os.path.join(_HERE, "csrc", "*.cu")))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a (one translation unit per file, in parallel) and link
    ``_build/librpa.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = _sources()
    deps = srcs + glob.glob(os.path.join(_HERE, "csrc", "*.cuh")) + [
        os.path.join(_ROOT, "include", "rpa.h")]
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(d) for d in deps)):
        return _SO
    nvcc = os.environ.get("NVCC", "nvcc")
    common = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I" + os.path.join(_ROOT, "include")]
    # extra compile definitions for variant builds, e.g. RPA_NVCC_FLAGS=-DRPA_DOT_F64=1
    common += os.environ.get("RPA_NVCC_FLAGS", "").split()

    def compile_one(src):
        obj = os.path.join(_BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = common + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = _SO + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, ARCH, "-shared", "-cudart=static", "-o", tmp] + objs,
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, _SO)
    return _SO


class Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("h", C.c_double * 3), ("bc", C.c_int * 3),
                ("fd_radius", C.c_int)]


class Options(C.Structure):
    _fields_ = [("lanczos_max", C.c_int), ("lanczos_rtol", C.c_double), ("stern_tol", C.c_double),
                ("stern_maxit", C.c_int), ("precision", C.c_int), ("reorth", C.c_int),
                ("stride", C.c_int * 3), ("interp", C.c_int), ("batch", C.c_int),
                ("fkind", C.c_int), ("refine", C.c_int), ("inner_tol", C.c_double),
                ("profile", C.c_int), ("tile", C.c_int), ("graphs", C.c_int),
                ("lanczos_block", C.c_int), ("refine_restart", C.c_int),
                ("debug_expire_waits", C.c_int), ("lanes", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("seconds_total", C.c_double), ("seconds_phase", C.c_double * 8),
                ("probe_points", C.c_longlong), ("matvecs", C.c_longlong),
                ("solves", C.c_longlong), ("cocg_iters", C.c_longlong),
                ("refine_rounds", C.c_longlong), ("max_cocg_iters", C.c_int),
                ("lanczos_steps_max", C.c_int), ("kernel_seconds", C.c_double * 8),
                ("kernel_launches", C.c_longlong * 8), ("kernel_bytes", C.c_double * 8),
                ("precision_bytes", C.c_int), ("tile_rows", C.c_int),
                ("tile_rows_tail", C.c_int), ("nonconv_solves", C.c_longlong),
                ("breakdown_solves", C.c_longlong)]

    def as_dict(self):
        return dict(seconds_total=self.seconds_total, seconds_phase=list(self.seconds_phase),
                    probe_points=self.probe_points, matvecs=self.matvecs, solves=self.solves,
                    cocg_iters=self.cocg_iters, refine_rounds=self.refine_rounds,
                    max_cocg_iters=self.max_cocg_iters,
                    lanczos_steps_max=self.lanczos_steps_max,
                    kernel_seconds=list(self.kernel_seconds),
                    kernel_launches=list(self.kernel_launches),
                    kernel_bytes=list(self.kernel_bytes),
                    precision_bytes=self.precision_bytes, tile_rows=self.tile_rows,
                    tile_rows_tail=self.tile_rows_tail, nonconv_solves=self.nonconv_solves,
                    breakdown_solves=self.breakdown_solves)


def _declare(lib):
    P, I, D, LL = C.c_void_p, C.c_int, C.c_double, C.c_longlong
    sig = {
        "rpa_create": ([P, P, P], I),
        "rpa_destroy": ([P], None),
        "rpa_set_potential": ([P, P, I], I),
        "rpa_set_projectors": ([P, I, P, P, P, P, P], I),
        "rpa_set_occupied": ([P, I, P, P, I], I),
        "rpa_set_frequencies": ([P, I, P, P], I),
        "rpa_gl_frequencies": ([I, P, P], I),
        "rpa_default_options": ([P], I),
        "rpa_set_options": ([P, P], I),
        "rpa_num_probes": ([P, P], I),
        "rpa_probe_indices": ([P, P], I),
        "rpa_energy_density": ([P, P, P, P, P, I], I),
        "rpa_probe_density": ([P, I, P, P, P, P, P, P, P, I], I),
        "rpa_interpolate": ([P, P, P, P, I], I),
        "rpa_apply_h": ([P, I, P, P, P, I], I),
        "rpa_apply_nu_half": ([P, I, P, P, I], I),
        "rpa_chi0": ([P, I, P, P, P, P, I], I),
        "rpa_tridiag_f11": ([I, I, P, P, I, P], I),
        "rpa_galerkin": ([P, I, P, P, P, I], I),
        "rpa_batch_energy": ([I, P, P, P], I),
        "rpa_set_checkpoint": ([P, C.c_char_p], I),
        "rpa_galerkin_noalloc": ([LL, I, P, P, D, I, P, P, P, P], I),
        "rpa_status_string": ([I], C.c_char_p),
        "rpa_last_error": ([P], C.c_char_p),
        "rpa_kernel_launches": ([P], LL),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


def load():
    """Load ``_build/librpa.so`` (build it first if absent).  Raises if it cannot be loaded."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            so = _SO if os.path.exists(_SO) else build()
            _LIB = _declare(C.CDLL(so))
    return _LIB


def header_symbols():
    """Names of the functions declared in include/rpa.h."""
    import re
    txt = open(os.path.join(_ROOT, "include", "rpa.h")).read()
    return sorted(set(re.findall(r"\b(rpa_[a-z0-9_]+)\s*\(", txt)))


# -------------------------------------------------------------------------------------------
# marshalling helpers
# -------------------------------------------------------------------------------------------
def _is_dev(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _ptr(a, dtype=None):
    if a is None:
        return None, None
    if _is_dev(a):
        return C.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=dtype) if dtype is not None else np.ascontiguousarray(a)
    return C.c_void_p(arr.ctypes.data), arr


def _where(*arrs):
    dev = [_is_dev(a) for a in arrs if a is not None]
    if dev and any(dev) and not all(dev):
        raise ValueError("all array arguments of one call must be host (numpy) or device (CUDA)")
    return RPA_DEVICE if (dev and dev[0]) else RPA_HOST


def _check(st, ctx=None):
    if st != RPA_OK:
        lib = load()
        msg = lib.rpa_last_error(ctx).decode() if ctx else ""
        if not msg:
            msg = lib.rpa_status_string(st).decode()
        raise RpaError(st, msg)


def _out(shape, dtype, like):
    if like is not None and _is_dev(like):
        import torch
        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64}[dtype]
        return torch.empty(shape, dtype=tdt, device=like.device)
    return np.empty(shape, dtype=dtype)


# -------------------------------------------------------------------------------------------
# the C entry points (same names)
# -------------------------------------------------------------------------------------------
def rpa_create(n, h, bc, fd_radius=6, stream=None):
    g = Grid()
    g.n[:] = [int(v) for v in n]
    g.h[:] = [float(v) for v in h]
    g.bc[:] = [int(v) for v in bc]
    g.fd_radius = int(fd_radius)
    out = C.c_void_p()
    st = load().rpa_create(C.byref(out), C.byref(g), C.c_void_p(stream) if stream else None)
    _check(st)
    return out


def rpa_destroy(ctx):
    if ctx:
        load().rpa_destroy(ctx)


def rpa_set_potential(ctx, vloc):
    p, keep = _ptr(vloc, np.float64)
    _check(load().rpa_set_potential(ctx, p, _where(vloc)), ctx)


def rpa_set_projectors(ctx, groups):
    """groups: iterable of (idx int[nnz], chi float[nproj, nnz], gamma float[nproj])."""
    groups = list(groups)
    if not groups:
        _check(load().rpa_set_projectors(ctx, 0, None, None, None, None, None), ctx)
        return
    nnz = np.array([len(g[0]) for g in groups], dtype=np.int32)
    npj = np.array([np.asarray(g[1]).shape[0] for g in groups], dtype=np.int32)
    idx = np.ascontiguousarray(np.concatenate([np.asarray(g[0], dtype=np.int32) for g in groups]))
    chi = np.ascontiguousarray(np.concatenate([np.asarray(g[1], dtype=np.float64).ravel() for g in groups]))
    gam = np.ascontiguousarray(np.concatenate([np.asarray(g[2], dtype=np.float64) for g in groups]))
    _check(load().rpa_set_projectors(ctx, len(groups), _ptr(nnz)[0], _ptr(npj)[0], _ptr(idx)[0],
                                     _ptr(chi)[0], _ptr(gam)[0]), ctx)


def rpa_set_occupied(ctx, psi, eps):
    ns = psi.shape[0]
    pp, k1 = _ptr(psi, np.float64)
    pe, k2 = _ptr(eps, np.float64)
    _check(load().rpa_set_occupied(ctx, ns, pp, pe, _where(psi, eps)), ctx)


def rpa_set_frequencies(ctx, omega, weight):
    om = np.ascontiguousarray(omega, dtype=np.float64)
    w = np.ascontiguousarray(weight, dtype=np.float64)
    _check(load().rpa_set_frequencies(ctx, len(om), _ptr(om)[0], _ptr(w)[0]), ctx)


def rpa_gl_frequencies(nw):
    om = np.empty(nw)
    w = np.empty(nw)
    _check(load().rpa_gl_frequencies(int(nw), _ptr(om)[0], _ptr(w)[0]))
    return om, w


def rpa_default_options():
    o = Options()
    _check(load().rpa_default_options(C.byref(o)))
    return o


def rpa_set_options(ctx, opts=None, **kw):
    o = opts if opts is not None else rpa_default_options()
    for k, v in kw.items():
        if k == "stride":
            o.stride[:] = [int(s) for s in v]
        elif k == "interp" and isinstance(v, str):
            o.interp = INTERP[v]
        elif k == "precision" and isinstance(v, str):
            o.precision = {"fp64": RPA_FP64, "mixed": RPA_MIXED,
                           "mixed_bf16": RPA_MIXED_BF16}[v]
        else:
            setattr(o, k, v)
    _check(load().rpa_set_options(ctx, C.byref(o)), ctx)
    return o


def rpa_num_probes(ctx):
    P = C.c_longlong()
    _check(load().rpa_num_probes(ctx, C.byref(P)), ctx)
    return P.value


def rpa_probe_indices(ctx):
    P = rpa_num_probes(ctx)
    out = np.empty(P, dtype=np.int64)
    _check(load().rpa_probe_indices(ctx, _ptr(out)[0]), ctx)
    return out


def rpa_energy_density(ctx, nw, nprobe, nd, device_like=None, want_fine=True):
    """Returns (d_coarse (nw x P), d_fine (nw x N_d) or None, E_c, stats dict)."""
    dco = _out((nw, nprobe), np.float64, device_like)
    dfi = _out((nw, nd), np.float64, device_like) if want_fine else None
    ec = _out((1,), np.float64, device_like)
    st = Stats()
    _check(load().rpa_energy_density(ctx, _ptr(dco)[0], _ptr(dfi)[0] if dfi is not None else None,
                                     _ptr(ec)[0], C.byref(st), _where(dco, dfi, ec)), ctx)
    return dco, dfi, float(ec[0]), st.as_dict()


def rpa_set_checkpoint(ctx, path):
    """Checkpoint file of rpa_energy_density (None turns it off)."""
    _check(load().rpa_set_checkpoint(ctx, os.fsencode(path) if path else None), ctx)


def rpa_probe_density(ctx, probes, freqs, nl=None, want_tridiag=False, device_like=None,
                      allow_nonconv=False):
    """Lanczos quadrature for explicit (probe, frequency-index) pairs.  Returns a dict."""
    if _is_dev(probes):
        pr, fq = probes, freqs
    else:
        pr = np.ascontiguousarray(probes, dtype=np.int64)
        fq = np.ascontiguousarray(freqs, dtype=np.int32)
    cnt = len(pr)
    d = _out((cnt,), np.float64, device_like if device_like is not None else pr)
    al = be = sp = None
    if want_tridiag:
        al = _out((cnt, nl), np.float64, d)
        be = _out((cnt, nl), np.float64, d)
        sp = _out((cnt,), np.int32, d)
    st = Stats()
    rc = load().rpa_probe_density(ctx, cnt, _ptr(pr)[0], _ptr(fq)[0], _ptr(d)[0],
                                  _ptr(al)[0] if al is not None else None,
                                  _ptr(be)[0] if be is not None else None,
                                  _ptr(sp)[0] if sp is not None else None, C.byref(st),
                                  _where(pr, fq, d))
    if not (allow_nonconv and rc == RPA_ENOCONV):
        _check(rc, ctx)
    return dict(d=d, alpha=al, beta=be, steps=sp, stats=st.as_dict(), status=rc)


def rpa_batch_energy(ctxs):
    """E_c of several contexts in one call (each on its own stream and host thread)."""
    n = len(ctxs)
    arr = (C.c_void_p * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    ec = np.zeros(n)
    st = (Stats * n)()
    rc = load().rpa_batch_energy(n, C.cast(arr, C.c_void_p), _ptr(ec)[0], C.cast(st, C.c_void_p))
    _check(rc, ctxs[0] if n else None)
    return ec, [s.as_dict() for s in st]


def rpa_interpolate(ctx, d_coarse, nd):
    dco = d_coarse
    nw = dco.shape[0]
    dfi = _out((nw, nd), np.float64, dco)
    ec = _out((1,), np.float64, dco)
    pc, keep = _ptr(dco, np.float64)
    _check(load().rpa_interpolate(ctx, pc, _ptr(dfi)[0], _ptr(ec)[0], _where(dco, dfi, ec)), ctx)
    return dfi, float(ec[0])


def rpa_apply_h(ctx, x, sigma):
    """x: complex (count, N_d); sigma: complex (count,).  Host numpy arrays."""
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.complex128)
    sg = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma, dtype=np.complex128), (x.shape[0],)))
    y = np.empty_like(x)
    _check(load().rpa_apply_h(ctx, x.shape[0], _ptr(x)[0], _ptr(sg)[0], _ptr(y)[0], RPA_HOST), ctx)
    return y


def rpa_apply_nu_half(ctx, q):
    q = np.ascontiguousarray(np.atleast_2d(q), dtype=np.float64)
    u = np.empty_like(q)
    _check(load().rpa_apply_nu_half(ctx, q.shape[0], _ptr(q)[0], _ptr(u)[0], RPA_HOST), ctx)
    return u


def rpa_chi0(ctx, omega, u, ns):
    u = np.ascontiguousarray(np.atleast_2d(u), dtype=np.float64)
    om = np.ascontiguousarray(np.broadcast_to(np.asarray(omega, dtype=np.float64), (u.shape[0],)))
    r = np.empty_like(u)
    it = np.zeros((u.shape[0], ns), dtype=np.int32)
    _check(load().rpa_chi0(ctx, u.shape[0], _ptr(om)[0], _ptr(u)[0], _ptr(r)[0], _ptr(it)[0],
                           RPA_HOST), ctx)
    return r, it


def rpa_galerkin(ctx, omega, u, ns):
    """Galerkin initial guesses x0 (count, ns, N_d) complex for (omega_i, u_i)."""
    u = np.ascontiguousarray(np.atleast_2d(u), dtype=np.float64)
    om = np.ascontiguousarray(np.broadcast_to(np.asarray(omega, dtype=np.float64), (u.shape[0],)))
    x0 = np.empty((u.shape[0], ns, u.shape[1]), dtype=np.complex128)
    _check(load().rpa_galerkin(ctx, u.shape[0], _ptr(om)[0], _ptr(u)[0], _ptr(x0)[0], RPA_HOST),
           ctx)
    return x0


# Scratch size of rpa_galerkin_noalloc (bytes); see include/rpa.h.
NOALLOC_SCRATCH_BYTES = 8 << 20


def _noalloc_check(psi, eps, omega, u, x0, stream):
    """Argument checks of rpa_galerkin_noalloc, all before the C call: the kernels take raw
    pointers and sizes, so a wrong dtype, shape, layout or device would make them read or
    write past the caller's buffers."""
    import torch
    args = dict(psi=psi, eps=eps, omega=omega, u=u, x0=x0)
    for k, t in args.items():
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"rpa_galerkin_noalloc: {k} must be a torch tensor")
    for k in ("psi", "eps", "omega", "u"):
        if args[k].dtype != torch.float64:
            raise ValueError(f"rpa_galerkin_noalloc: {k} must be float64, got {args[k].dtype}")
    if x0.dtype != torch.complex128:
        raise ValueError(f"rpa_galerkin_noalloc: x0 must be complex128, got {x0.dtype}")
    if psi.dim() != 2 or u.dim() != 2 or eps.dim() != 1 or omega.dim() != 1 or x0.dim() != 3:
        raise ValueError("rpa_galerkin_noalloc: expected psi (ns, nd), eps (ns,), omega (count,), "
                         "u (count, nd), x0 (count, ns, nd)")
    ns, nd = int(psi.shape[0]), int(psi.shape[1])
    count = int(u.shape[0])
    want = dict(eps=(ns,), omega=(count,), u=(count, nd), x0=(count, ns, nd))
    for k, shp in want.items():
        if tuple(args[k].shape) != shp:
            raise ValueError(f"rpa_galerkin_noalloc: {k} has shape {tuple(args[k].shape)}, "
                             f"expected {shp}")
    for k, t in args.items():
        if not t.is_contiguous():
            raise ValueError(f"rpa_galerkin_noalloc: {k} must be contiguous")
    dev = psi.device
    for k, t in args.items():
        if not t.is_cuda or t.device != dev:
            raise ValueError(f"rpa_galerkin_noalloc: {k} must be a CUDA tensor on {dev}")
    if dev.index != torch.cuda.current_device():
        raise ValueError("rpa_galerkin_noalloc: the tensors must live on the current device")
    if stream is not None and getattr(stream, "device", dev) != dev:
        raise ValueError("rpa_galerkin_noalloc: the stream belongs to another device")


def rpa_galerkin_noalloc(psi, eps, dV, omega, u, x0, stream=None):
    """FP64 Galerkin guesses for callers that cannot allocate device memory.

    All arguments are contiguous CUDA tensors on the current device, owned by the caller:
    psi (ns, nd) float64, eps (ns,) float64, omega (count,) float64, u (count, nd) float64,
    x0 (count, ns, nd) complex128 output; anything else raises ValueError before any work is
    queued.  Work is queued on `stream` (a torch.cuda.Stream or None for the current stream)
    without synchronising.  Uses a fixed 8 MiB device scratch array inside the library; sizes
    beyond it raise RpaError(RPA_EINVAL)."""
    import torch
    _noalloc_check(psi, eps, omega, u, x0, stream)
    ns, nd = int(psi.shape[0]), int(psi.shape[1])
    count = int(u.shape[0])
    nchunk = min(256, max(1, (nd + 4095) // 4096))
    need = ((nchunk * ns * ns * 8 + 255) // 256) * 256 + ns * ns * 16
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = load().rpa_galerkin_noalloc(nd, ns, C.c_void_p(psi.data_ptr()),
                                     C.c_void_p(eps.data_ptr()), float(dV), count,
                                     C.c_void_p(omega.data_ptr()), C.c_void_p(u.data_ptr()),
                                     C.c_void_p(x0.data_ptr()), C.c_void_p(st.cuda_stream))
    if rc == RPA_EINVAL and need > NOALLOC_SCRATCH_BYTES:
        raise RpaError(rc, f"rpa_galerkin_noalloc: needs {need} bytes of scratch, more than "
                           f"the {NOALLOC_SCRATCH_BYTES} bytes it holds")
    _check(rc)
    return x0


def rpa_tridiag_f11(alpha, beta, fkind=RPA_F_LOG):
    a = np.ascontiguousarray(np.atleast_2d(alpha), dtype=np.float64)
    b = np.ascontiguousarray(np.atleast_2d(beta), dtype=np.float64)
    cnt, k = a.shape
    if b.shape[1] < k:
        b = np.ascontiguousarray(np.pad(b, ((0, 0), (0, k - b.shape[1]))))
    d = np.empty(cnt)
    _check(load().rpa_tridiag_f11(cnt, k, _ptr(a)[0], _ptr(b)[0], int(fkind), _ptr(d)[0]))
    return d


def rpa_kernel_launches(ctx=None):
    return int(load().rpa_kernel_launches(ctx))


# -------------------------------------------------------------------------------------------
# convenience: a context set up from arrays describing one system
# -------------------------------------------------------------------------------------------
class Context:
    """Owns one rpa_ctx; ``setup`` feeds grid, potential, projectors, occupied pairs."""

    def __init__(self, n, h, bc, fd_radius=6, stream=None):
        self.ctx = rpa_create(n, h, bc, fd_radius, stream)
        self.n, self.h, self.bc = tuple(n), tuple(h), tuple(bc)
        self.nd = int(np.prod(n))

    def close(self):
        if self.ctx:
            rpa_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @classmethod
    def from_system(cls, s, omega=None, weight=None, **opts):
        c = cls(s.n, s.h, s.bc, s.fd_radius)
        rpa_set_potential(c.ctx, s.vloc)
        rpa_set_projectors(c.ctx, [(g.idx, g.chi, g.gamma) for g in s.groups])
        rpa_set_occupied(c.ctx, s.psi, s.eps)
        if omega is not None:
            rpa_set_frequencies(c.ctx, omega, weight)
        c.opts = rpa_set_options(c.ctx, **opts) if opts else rpa_set_options(c.ctx)
        c.ns = s.psi.shape[0]
        return c
