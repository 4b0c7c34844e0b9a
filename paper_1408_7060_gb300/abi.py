"""ctypes binding of ``libaim_gb300.so`` (the C ABI in ``include/aim.h``).

Argument marshalling only: every computation runs in the CUDA library.  Arrays may
be numpy arrays (host) or torch tensors (host or CUDA); complex arrays are
complex128 with shape ``[nb, ns]`` (``[steps, nb, ns]`` for histories and marches).
Functions keep the C names (``aim_setup``, ``aim_matvec``, ...); ``AimContext`` is
a convenience wrapper around them.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from . import build as _build

AIM_OK, AIM_ERR_ARG, AIM_ERR_MESH, AIM_ERR_CUDA, AIM_ERR_OOM, AIM_ERR_NOCONV, AIM_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
AIM_WARN_UNSTABLE = 1
AIM_C128, AIM_C64 = 0, 1
AIM_CPPIF = 0
AIM_BLIF = 1
AIM_PLAN_DEFAULT, AIM_PLAN_MEASURED, AIM_PLAN_CACHED = 0, 1, 2

_NAMES = {0: "AIM_OK", -1: "AIM_ERR_ARG", -2: "AIM_ERR_MESH", -3: "AIM_ERR_CUDA", -4: "AIM_ERR_OOM",
          -5: "AIM_ERR_NOCONV", -6: "AIM_ERR_TIMEOUT", 1: "AIM_WARN_UNSTABLE"}


class AimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class aim_mesh(ct.Structure):
    _fields_ = [("nv", ct.c_int32), ("nt", ct.c_int32), ("v", ct.c_void_p), ("tri", ct.c_void_p)]


class aim_grid(ct.Structure):
    _fields_ = [("n", ct.c_int32), ("origin", ct.c_double * 3), ("h", ct.c_double)]


class aim_tbasis(ct.Structure):
    _fields_ = [("kind", ct.c_int32), ("order", ct.c_int32)]


class aim_opts(ct.Structure):
    _fields_ = [("f_c", ct.c_double), ("precision", ct.c_int32), ("batch_max", ct.c_int32),
                ("gmres_restart", ct.c_int32), ("gmres_max_iter", ct.c_int32), ("cuda_stream", ct.c_void_p),
                ("preconditioner", ct.c_int32), ("precond_radius", ct.c_double), ("zero_start", ct.c_int32),
                ("refine", ct.c_int32), ("refine_every", ct.c_int32), ("autotune", ct.c_int32),
                ("rhs_blocked", ct.c_int32), ("eps_r", ct.c_double), ("mu_r", ct.c_double),
                ("blif_band", ct.c_double)]


class aim_excitation(ct.Structure):
    _fields_ = [("nb", ct.c_int32), ("khat", ct.c_void_p), ("phat", ct.c_void_p),
                ("sigma", ct.c_double), ("t_d", ct.c_double)]


class aim_stats(ct.Structure):
    _fields_ = [("last_step", ct.c_int32), ("total_iters", ct.c_int32), ("max_iters", ct.c_int32),
                ("max_rel_res", ct.c_double), ("rhs_ms", ct.c_double), ("solve_ms", ct.c_double),
                ("iters", ct.c_void_p), ("refine_corrections", ct.c_int32), ("refine_checks", ct.c_int32)]


class aim_info(ct.Structure):
    _fields_ = [("ns", ct.c_int32), ("n_delays", ct.c_int32), ("n_active", ct.c_int32),
                ("near_nnz", ct.c_int64), ("grid_n", ct.c_int32), ("precision", ct.c_int32),
                ("device_bytes", ct.c_int64), ("preconditioner", ct.c_int32), ("precond_nnz", ct.c_int64),
                ("refine", ct.c_int32), ("refine_every", ct.c_int32), ("plan_zw", ct.c_int32), ("plan_cw", ct.c_int32), ("plan_rp", ct.c_int32),
                ("plan_ypb", ct.c_int32), ("plan_source", ct.c_int32), ("box_lo", ct.c_int32 * 3),
                ("box_hi", ct.c_int32 * 3), ("rhs_blocked", ct.c_int32), ("z_len", ct.c_int32)]


EXPORTS = ["aim_setup", "aim_destroy", "aim_last_error", "aim_get_info", "aim_time_factor", "aim_num_unknowns", "aim_rwg_table",
           "aim_matvec", "aim_rhs", "aim_excitation_vector", "aim_march", "aim_march_continue", "aim_get_anterp",
           "aim_get_near", "aim_get_preconditioner", "aim_get_kernel_spectrum", "aim_profile", "aim_get_profile", "aim_kernel_name",
           "aim_matvec_noalloc", "aim_march_source", "aim_excitation_samples", "aim_excitation_samples_adjoint",
           "aim_farfield", "aim_farfield_adjoint", "aim_march_adjoint", "aim_march_farfield",
           "aim_march_adjoint_farfield", "aim_march_spectrum", "aim_rcs"]
AIM_K_COUNT = 15

_LIB = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ct.CDLL:
    """Load the CUDA library (building it in-tree first if it is missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library {_build.LIB} is missing; run __graft_entry__.build()")
    lib = ct.CDLL(_build.LIB)
    P, I32, D = ct.c_void_p, ct.c_int32, ct.c_double
    sig = {
        "aim_setup": (ct.c_int, [ct.POINTER(aim_mesh), ct.POINTER(aim_grid), D, D, aim_tbasis,
                                 ct.POINTER(aim_opts), ct.POINTER(P)]),
        "aim_destroy": (None, [P]),
        "aim_last_error": (ct.c_char_p, [P]),
        "aim_get_info": (ct.c_int, [P, ct.POINTER(aim_info)]),
        "aim_time_factor": (ct.c_int, [aim_tbasis, D, I32, I32, ct.c_void_p, ct.c_void_p]),
        "aim_num_unknowns": (ct.c_int, [P, ct.POINTER(I32), ct.POINTER(I32)]),
        "aim_rwg_table": (ct.c_int, [P, P, P, P]),
        "aim_matvec": (ct.c_int, [P, I32, I32, P, P]),
        "aim_rhs": (ct.c_int, [P, I32, I32, P, P]),
        "aim_matvec_noalloc": (ct.c_int, [P, I32, I32, P, P]),
        "aim_excitation_vector": (ct.c_int, [P, ct.POINTER(aim_excitation), I32, P]),
        "aim_march": (ct.c_int, [P, ct.POINTER(aim_excitation), I32, D, P, ct.POINTER(aim_stats)]),
        "aim_march_continue": (ct.c_int, [P, ct.POINTER(aim_excitation), I32, D, P, ct.POINTER(aim_stats)]),
        "aim_profile": (ct.c_int, [P, I32]),
        "aim_get_profile": (ct.c_int, [P, P, P, P]),
        "aim_kernel_name": (ct.c_char_p, [I32]),
        "aim_march_source": (ct.c_int, [P, I32, I32, I32, P, D, P, ct.POINTER(aim_stats)]),
        "aim_excitation_samples": (ct.c_int, [P, P, P, I32, I32, P, I32, P]),
        "aim_excitation_samples_adjoint": (ct.c_int, [P, P, P, I32, I32, I32, P, P]),
        "aim_farfield": (ct.c_int, [P, I32, P, P, P, I32, P, I32, I32, P]),
        "aim_farfield_adjoint": (ct.c_int, [P, I32, P, P, P, I32, I32, I32, P, P]),
        "aim_march_adjoint": (ct.c_int, [P, I32, I32, P, D, P, ct.POINTER(aim_stats)]),
        "aim_march_farfield": (ct.c_int, [P, P, P, I32, I32, P, I32, D, I32, P, P, P, I32, I32, P,
                                          ct.POINTER(aim_stats)]),
        "aim_march_adjoint_farfield": (ct.c_int, [P, P, P, I32, I32, I32, D, I32, P, P, P, I32, I32, P, P,
                                                  ct.POINTER(aim_stats)]),
        "aim_march_spectrum": (ct.c_int, [P, ct.POINTER(aim_excitation), I32, D, I32, P, P, ct.POINTER(aim_stats)]),
        "aim_rcs": (ct.c_int, [P, I32, P, I32, P, I32, P, P, P]),
        "aim_get_anterp": (ct.c_int, [P, P, P]),
        "aim_get_near": (ct.c_int, [P, P, P, P]),
        "aim_get_preconditioner": (ct.c_int, [P, P, P, P]),
        "aim_get_kernel_spectrum": (ct.c_int, [P, I32, I32, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


# ----------------------------------------------------------------------------- marshalling

def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (contiguous)."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    raise TypeError(type(a))


def _like(x, shape):
    """An output complex128 array of ``shape`` on the same side (numpy / torch device) as x."""
    if isinstance(x, np.ndarray):
        return np.empty(shape, dtype=np.complex128)
    import torch

    return torch.empty(shape, dtype=torch.complex128, device=x.device)


def _check(lib, ctx, rc, what, stats=None):
    if rc < 0:
        msg = lib.aim_last_error(ctx)
        err = AimError(rc, f"{what}: {msg.decode() if msg else ''}")
        err.stats = stats   # march statistics (AIM_ERR_NOCONV: steps up to last_step are valid)
        raise err
    return rc


def _stats(st, iters):
    out = {f: getattr(st, f) for f, _ in aim_stats._fields_ if f != "iters"}
    out["iters"] = iters
    return out


def _stream_handle():
    try:
        import torch

        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


PRECOND = {"diag": 0, "sai": 1}  # AIM_PRECOND_DIAG, AIM_PRECOND_NEAR_SAI


def aim_setup(V, F, grid_n, origin, h, near_radius, dt, f_c, order=2, precision="c64", batch_max=1,
              restart=50, max_iter=500, stream=None, precond="diag", precond_radius=0.0, zero_start=False,
              refine=0, autotune=0, refine_every=1, rhs_blocked=0, eps_r=1.0, mu_r=1.0, basis="cppif",
              blif_band=0.25):
    """Build a context; returns an opaque handle (int).  precond: "diag" (the paper's
    diagonal preconditioner) or "sai" (sparse approximate inverse on the pairs within
    precond_radius, default the near radius).  zero_start: GMRES from zero instead of
    the previous step's currents.  refine (complex64 only): up to this many FP64
    refinement corrections per step (0: off), checked every refine_every-th step.
    autotune: 0 default launch shapes, 1 tuned at setup (cached plan reused), 2 tuned and
    cache refreshed.  rhs_blocked: delayed grid sums by the multilevel blocked schedule
    (power-of-two z transforms).  eps_r, mu_r: the homogeneous background medium.  basis:
    "cppif" (order = Q) or "blif" (order = the half-width M, blif_band = f_bw dt)."""
    lib = load()
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    mesh = aim_mesh(len(V), len(F), V.ctypes.data, F.ctypes.data)
    grid = aim_grid(int(grid_n), (ct.c_double * 3)(*[float(o) for o in origin]), float(h))
    tb = aim_tbasis({"cppif": AIM_CPPIF, "blif": AIM_BLIF}[basis], int(order))
    prec = {"c128": AIM_C128, "c64": AIM_C64}[precision]
    opts = aim_opts(float(f_c), prec, int(batch_max), int(restart), int(max_iter),
                    stream if stream is not None else _stream_handle(), PRECOND[precond], float(precond_radius),
                    int(bool(zero_start)), int(refine), int(refine_every), int(autotune), int(bool(rhs_blocked)),
                    float(eps_r), float(mu_r), float(blif_band))
    out = ct.c_void_p()
    rc = lib.aim_setup(ct.byref(mesh), ct.byref(grid), float(near_radius), float(dt), tb, ct.byref(opts),
                       ct.byref(out))
    _check(lib, None, rc, "aim_setup")
    return out.value


def aim_destroy(ctx):
    load().aim_destroy(ctx)


def aim_get_info(ctx) -> dict:
    lib = load()
    info = aim_info()
    _check(lib, ctx, lib.aim_get_info(ctx, ct.byref(info)), "aim_get_info")
    out = {f: getattr(info, f) for f, _ in aim_info._fields_}
    out["box_lo"], out["box_hi"] = tuple(info.box_lo), tuple(info.box_hi)
    return out


def aim_time_factor(m, x, basis="cppif", order=2, blif_band=0.25):
    """[len(x), 4]: the time factor of delay m and its first three derivatives at x = R/(c dt)
    (host computation, no GPU)."""
    lib = load()
    x = np.ascontiguousarray(np.atleast_1d(x), dtype=np.float64)
    out = np.zeros((len(x), 4))
    tb = aim_tbasis({"cppif": AIM_CPPIF, "blif": AIM_BLIF}[basis], int(order))
    _check(lib, None, lib.aim_time_factor(tb, float(blif_band), int(m), len(x), x.ctypes.data, out.ctypes.data),
           "aim_time_factor")
    return out


def aim_num_unknowns(ctx):
    lib = load()
    ns, ng = ct.c_int32(), ct.c_int32()
    _check(lib, ctx, lib.aim_num_unknowns(ctx, ct.byref(ns), ct.byref(ng)), "aim_num_unknowns")
    return ns.value, ng.value


def aim_rwg_table(ctx):
    lib = load()
    ns, _ = aim_num_unknowns(ctx)
    e, t, f = (np.empty((ns, 2), dtype=np.int32) for _ in range(3))
    _check(lib, ctx, lib.aim_rwg_table(ctx, e.ctypes.data, t.ctypes.data, f.ctypes.data), "aim_rwg_table")
    return e, t, f


def aim_matvec(ctx, m, x, out=None):
    """y = Z~AIM_m x for x[nb, ns] complex128 (numpy or torch)."""
    lib = load()
    y = _like(x, tuple(x.shape)) if out is None else out
    _check(lib, ctx, lib.aim_matvec(ctx, int(m), int(x.shape[0]), _ptr(x), _ptr(y)), "aim_matvec")
    return y


def aim_matvec_noalloc(ctx, m, x, out=None):
    """aim_matvec with the grid work space in the library's fixed device array."""
    lib = load()
    y = _like(x, tuple(x.shape)) if out is None else out
    _check(lib, ctx, lib.aim_matvec_noalloc(ctx, int(m), int(x.shape[0]), _ptr(x), _ptr(y)), "aim_matvec_noalloc")
    return y


def aim_rhs(ctx, step_l, hist, out=None):
    """sum_{m>=1} Z~AIM_m I_{l-m} for hist[N_g, nb, ns] with hist[m-1] = I_{l-m}."""
    lib = load()
    y = _like(hist, tuple(hist.shape[1:])) if out is None else out
    _check(lib, ctx, lib.aim_rhs(ctx, int(step_l), int(hist.shape[1]), _ptr(hist), _ptr(y)), "aim_rhs")
    return y


def _exc(khat, phat, sigma, t_d):
    khat = np.ascontiguousarray(np.atleast_2d(khat), dtype=np.float64)
    phat = np.ascontiguousarray(np.atleast_2d(phat), dtype=np.float64)
    e = aim_excitation(len(khat), khat.ctypes.data, phat.ctypes.data, float(sigma), float(t_d))
    return e, (khat, phat)


def aim_excitation_vector(ctx, khat, phat, sigma, t_d, step_l, out=None):
    lib = load()
    ns, _ = aim_num_unknowns(ctx)
    e, keep = _exc(khat, phat, sigma, t_d)
    y = np.empty((e.nb, ns), dtype=np.complex128) if out is None else out
    _check(lib, ctx, lib.aim_excitation_vector(ctx, ct.byref(e), int(step_l), _ptr(y)), "aim_excitation_vector")
    return y


def aim_march(ctx, khat, phat, sigma, t_d, n_steps, tol, out=None):
    """March Eq. 5 for n_steps; returns (currents[n_steps, nb, ns], stats dict, status)."""
    lib = load()
    ns, _ = aim_num_unknowns(ctx)
    e, keep = _exc(khat, phat, sigma, t_d)
    cur = np.empty((n_steps, e.nb, ns), dtype=np.complex128) if out is None else out
    iters = np.zeros((n_steps, e.nb), dtype=np.int32)
    st = aim_stats(0, 0, 0, 0.0, 0.0, 0.0, iters.ctypes.data, 0, 0)
    rc = lib.aim_march(ctx, ct.byref(e), int(n_steps), float(tol), _ptr(cur), ct.byref(st))
    stats = _stats(st, iters)
    _check(lib, ctx, rc, "aim_march", stats)
    return cur, stats, rc


def aim_march_spectrum(ctx, khat, phat, sigma, t_d, n_steps, tol, freqs, out=None):
    """March Eq. 5 from rest and return the frequency-domain currents for a unit incident
    field at ``freqs`` (Hz): (spec[n_freq, nb, ns], stats dict, status)."""
    lib = load()
    ns, _ = aim_num_unknowns(ctx)
    e, keep = _exc(khat, phat, sigma, t_d)
    fr = np.ascontiguousarray(np.atleast_1d(freqs), dtype=np.float64)
    spec = np.empty((len(fr), e.nb, ns), dtype=np.complex128) if out is None else out
    iters = np.zeros((n_steps, e.nb), dtype=np.int32)
    st = aim_stats(0, 0, 0, 0.0, 0.0, 0.0, iters.ctypes.data, 0, 0)
    rc = lib.aim_march_spectrum(ctx, ct.byref(e), int(n_steps), float(tol), len(fr), fr.ctypes.data, _ptr(spec),
                                ct.byref(st))
    stats = _stats(st, iters)
    _check(lib, ctx, rc, "aim_march_spectrum", stats)
    return spec, stats, rc


def aim_rcs(ctx, freqs, spec, rhat, pol, out=None):
    """Bistatic RCS (m^2) of frequency-domain currents spec[n_freq, nb, ns] in the
    directions rhat[nd, 3] for receive polarisations pol[nd, 3]: [n_freq, nb, nd]."""
    lib = load()
    fr = np.ascontiguousarray(np.atleast_1d(freqs), dtype=np.float64)
    rh = np.ascontiguousarray(rhat, dtype=np.float64).reshape(-1, 3)
    po = np.ascontiguousarray(pol, dtype=np.float64).reshape(-1, 3)
    nb = spec.shape[1]
    sig = np.empty((len(fr), nb, len(rh))) if out is None else out
    _check(lib, ctx, lib.aim_rcs(ctx, len(fr), fr.ctypes.data, nb, _ptr(spec), len(rh), rh.ctypes.data,
                                 po.ctypes.data, _ptr(sig)), "aim_rcs")
    return sig


def aim_march_continue(ctx, khat, phat, sigma, t_d, n_steps, tol, out=None):
    """Advance the march started by aim_march on this context by n_steps."""
    lib = load()
    ns, _ = aim_num_unknowns(ctx)
    e, keep = _exc(khat, phat, sigma, t_d)
    cur = np.empty((n_steps, e.nb, ns), dtype=np.complex128) if out is None else out
    iters = np.zeros((n_steps, e.nb), dtype=np.int32)
    st = aim_stats(0, 0, 0, 0.0, 0.0, 0.0, iters.ctypes.data, 0, 0)
    rc = lib.aim_march_continue(ctx, ct.byref(e), int(n_steps), float(tol), _ptr(cur), ct.byref(st))
    stats = _stats(st, iters)
    _check(lib, ctx, rc, "aim_march_continue", stats)
    return cur, stats, rc


def aim_profile(ctx, enable=True):
    lib = load()
    _check(lib, ctx, lib.aim_profile(ctx, int(bool(enable))), "aim_profile")


def aim_get_profile(ctx) -> dict:
    """{kernel name: (launches, device ms)} and the total launch count."""
    lib = load()
    n = np.zeros(AIM_K_COUNT, dtype=np.int64)
    ms = np.zeros(AIM_K_COUNT, dtype=np.float64)
    tot = np.zeros(1, dtype=np.int64)
    _check(lib, ctx, lib.aim_get_profile(ctx, n.ctypes.data, ms.ctypes.data, tot.ctypes.data), "aim_get_profile")
    out = {lib.aim_kernel_name(i).decode(): (int(n[i]), float(ms[i])) for i in range(AIM_K_COUNT)}
    return out, int(tot[0])


def _vec3(x, n=None):
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    return x


def aim_march_source(ctx, src, tol, transpose=False, out=None):
    """March from rest with explicit right-hand sides src[n_steps, nb, ns]."""
    lib = load()
    n_steps, nb, ns = src.shape
    cur = _like(src, tuple(src.shape)) if out is None else out
    iters = np.zeros((n_steps, nb), dtype=np.int32)
    st = aim_stats(0, 0, 0, 0.0, 0.0, 0.0, iters.ctypes.data, 0, 0)
    rc = lib.aim_march_source(ctx, int(bool(transpose)), int(nb), int(n_steps), _ptr(src), float(tol), _ptr(cur),
                              ct.byref(st))
    stats = _stats(st, iters)
    _check(lib, ctx, rc, "aim_march_source", stats)
    return cur, stats, rc


def aim_march_adjoint(ctx, G, tol, out=None):
    """The adjoint march M^H lam = G for G[n_steps, nb, ns]; returns (lam, stats, status)."""
    lib = load()
    n_steps, nb, ns = G.shape
    lam = _like(G, tuple(G.shape)) if out is None else out
    iters = np.zeros((n_steps, nb), dtype=np.int32)
    st = aim_stats(0, 0, 0, 0.0, 0.0, 0.0, iters.ctypes.data, 0, 0)
    rc = lib.aim_march_adjoint(ctx, int(nb), int(n_steps), _ptr(G), float(tol), _ptr(lam), ct.byref(st))
    stats = _stats(st, iters)
    _check(lib, ctx, rc, "aim_march_adjoint", stats)
    return lam, stats, rc


def aim_march_farfield(ctx, khat, phat, i0, a, n_steps, tol, rhat, e1, e2, n0, n_out, out=None):
    """Far-field envelope F[n_out, nd, 2] of the march driven by envelope samples a (no
    current history is kept); returns (F, stats, status)."""
    lib = load()
    k, p = _vec3(khat), _vec3(phat)
    r, u, v = _vec3(rhat), _vec3(e1), _vec3(e2)
    F = _like(a, (int(n_out), len(r), 2)) if out is None else out
    iters = np.zeros((int(n_steps), 1), dtype=np.int32)
    st = aim_stats(0, 0, 0, 0.0, 0.0, 0.0, iters.ctypes.data, 0, 0)
    rc = lib.aim_march_farfield(ctx, k.ctypes.data, p.ctypes.data, int(i0), int(a.shape[0]), _ptr(a), int(n_steps),
                                float(tol), len(r), r.ctypes.data, u.ctypes.data, v.ctypes.data, int(n0),
                                int(n_out), _ptr(F), ct.byref(st))
    stats = _stats(st, iters)
    _check(lib, ctx, rc, "aim_march_farfield", stats)
    return F, stats, rc


def aim_march_adjoint_farfield(ctx, khat, phat, i0, n_samp, n_steps, tol, rhat, e1, e2, n0, F, out=None):
    """grad[n_samp] = B^H M^{-H} A^H F (dJ/d conj(a) of J = sum |F|^2); returns (grad, stats, status)."""
    lib = load()
    k, p = _vec3(khat), _vec3(phat)
    r, u, v = _vec3(rhat), _vec3(e1), _vec3(e2)
    g = _like(F, (int(n_samp),)) if out is None else out
    iters = np.zeros((int(n_steps), 1), dtype=np.int32)
    st = aim_stats(0, 0, 0, 0.0, 0.0, 0.0, iters.ctypes.data, 0, 0)
    rc = lib.aim_march_adjoint_farfield(ctx, k.ctypes.data, p.ctypes.data, int(i0), int(n_samp), int(n_steps),
                                        float(tol), len(r), r.ctypes.data, u.ctypes.data, v.ctypes.data, int(n0),
                                        int(F.shape[0]), _ptr(F), _ptr(g), ct.byref(st))
    stats = _stats(st, iters)
    _check(lib, ctx, rc, "aim_march_adjoint_farfield", stats)
    return g, stats, rc


def aim_excitation_samples(ctx, khat, phat, i0, a, n_steps, out=None):
    lib = load()
    ns, _ = aim_num_unknowns(ctx)
    k, p = _vec3(khat), _vec3(phat)
    V = _like(a, (int(n_steps), ns)) if out is None else out
    _check(lib, ctx, lib.aim_excitation_samples(ctx, k.ctypes.data, p.ctypes.data, int(i0), int(a.shape[0]), _ptr(a),
                                                int(n_steps), _ptr(V)), "aim_excitation_samples")
    return V


def aim_excitation_samples_adjoint(ctx, khat, phat, i0, n_samp, lam, out=None):
    lib = load()
    k, p = _vec3(khat), _vec3(phat)
    g = _like(lam, (int(n_samp),)) if out is None else out
    _check(lib, ctx, lib.aim_excitation_samples_adjoint(ctx, k.ctypes.data, p.ctypes.data, int(i0), int(n_samp),
                                                        int(lam.shape[0]), _ptr(lam), _ptr(g)),
           "aim_excitation_samples_adjoint")
    return g


def aim_farfield(ctx, rhat, e1, e2, I, n0, n_out, out=None):
    lib = load()
    r, a, b = _vec3(rhat), _vec3(e1), _vec3(e2)
    F = _like(I, (int(n_out), len(r), 2)) if out is None else out
    _check(lib, ctx, lib.aim_farfield(ctx, len(r), r.ctypes.data, a.ctypes.data, b.ctypes.data, int(I.shape[0]),
                                      _ptr(I), int(n0), int(n_out), _ptr(F)), "aim_farfield")
    return F


def aim_farfield_adjoint(ctx, rhat, e1, e2, n_steps, n0, F, out=None):
    lib = load()
    r, a, b = _vec3(rhat), _vec3(e1), _vec3(e2)
    ns, _ = aim_num_unknowns(ctx)
    G = _like(F, (int(n_steps), ns)) if out is None else out
    _check(lib, ctx, lib.aim_farfield_adjoint(ctx, len(r), r.ctypes.data, a.ctypes.data, b.ctypes.data,
                                              int(n_steps), int(n0), int(F.shape[0]), _ptr(F), _ptr(G)),
           "aim_farfield_adjoint")
    return G


def aim_get_anterp(ctx):
    lib = load()
    ns, _ = aim_num_unknowns(ctx)
    anchor = np.empty((ns, 3), dtype=np.int32)
    lam = np.empty((ns, 4, 64), dtype=np.float64)
    _check(lib, ctx, lib.aim_get_anterp(ctx, anchor.ctypes.data, lam.ctypes.data), "aim_get_anterp")
    return anchor, lam


def aim_get_near(ctx):
    lib = load()
    info = aim_get_info(ctx)
    ns, nnz, ng = info["ns"], info["near_nnz"], info["n_delays"]
    rowptr = np.empty(ns + 1, dtype=np.int32)
    col = np.empty(max(nnz, 1), dtype=np.int32)
    val = np.empty((ng + 1, max(nnz, 1)), dtype=np.complex128)
    _check(lib, ctx, lib.aim_get_near(ctx, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data), "aim_get_near")
    return rowptr, col[:nnz], val[:, :nnz]


def aim_get_preconditioner(ctx):
    """The right preconditioner M in CSR form (rowptr, col, val), val[e] = M[row, col[e]]."""
    lib = load()
    info = aim_get_info(ctx)
    ns, nnz = info["ns"], info["precond_nnz"]
    rowptr = np.empty(ns + 1, dtype=np.int32)
    col = np.empty(max(nnz, 1), dtype=np.int32)
    val = np.empty(max(nnz, 1), dtype=np.complex128)
    _check(lib, ctx, lib.aim_get_preconditioner(ctx, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data),
           "aim_get_preconditioner")
    return rowptr, col[:nnz], val[:nnz]


def aim_get_kernel_spectrum(ctx, m, kind):
    lib = load()
    info = aim_get_info(ctx)
    n = info["grid_n"] + 1
    out = np.empty((info["z_len"] // 2 + 1, n, n), dtype=np.complex128)
    _check(lib, ctx, lib.aim_get_kernel_spectrum(ctx, int(m), int(kind), out.ctypes.data), "aim_get_kernel_spectrum")
    return out


class AimContext:
    """Owning wrapper: ``with AimContext.from_workload(w) as ctx: ctx.matvec(0, x)``."""

    def __init__(self, **kw):
        self.handle = aim_setup(**kw)
        self.info = aim_get_info(self.handle)
        self.ns = self.info["ns"]
        self.n_delays = self.info["n_delays"]

    @classmethod
    def from_workload(cls, w, **over):
        V, F = w.mesh
        kw = dict(V=V, F=F, grid_n=w.grid_n, origin=w.origin, h=w.h, near_radius=w.near_radius, dt=w.dt,
                  f_c=w.f_c, order=w.order, precision=w.precision, batch_max=w.nb, precond=w.precond,
                  precond_radius=w.precond_radius, zero_start=w.zero_start, refine=w.refine,
                  refine_every=w.refine_every, autotune=w.autotune, rhs_blocked=w.rhs_blocked, eps_r=w.eps_r,
                  mu_r=w.mu_r, basis=w.basis, blif_band=w.beta)
        kw.update(over)
        return cls(**kw)

    def matvec(self, m, x, out=None):
        return aim_matvec(self.handle, m, x, out)

    def rhs(self, step_l, hist, out=None):
        return aim_rhs(self.handle, step_l, hist, out)

    def excitation(self, khat, phat, sigma, t_d, step_l):
        return aim_excitation_vector(self.handle, khat, phat, sigma, t_d, step_l)

    def march(self, khat, phat, sigma, t_d, n_steps, tol, out=None):
        return aim_march(self.handle, khat, phat, sigma, t_d, n_steps, tol, out)

    def march_spectrum(self, khat, phat, sigma, t_d, n_steps, tol, freqs, out=None):
        return aim_march_spectrum(self.handle, khat, phat, sigma, t_d, n_steps, tol, freqs, out)

    def rcs(self, freqs, spec, rhat, pol, out=None):
        return aim_rcs(self.handle, freqs, spec, rhat, pol, out)

    def march_continue(self, khat, phat, sigma, t_d, n_steps, tol, out=None):
        return aim_march_continue(self.handle, khat, phat, sigma, t_d, n_steps, tol, out)

    def profile(self, enable=True):
        aim_profile(self.handle, enable)

    def get_profile(self):
        return aim_get_profile(self.handle)

    def rwg_table(self):
        return aim_rwg_table(self.handle)

    def anterp(self):
        return aim_get_anterp(self.handle)

    def near(self):
        return aim_get_near(self.handle)

    def preconditioner(self):
        return aim_get_preconditioner(self.handle)

    def kernel_spectrum(self, m, kind):
        return aim_get_kernel_spectrum(self.handle, m, kind)

    def close(self):
        if self.handle:
            aim_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
