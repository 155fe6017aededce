"""Thin ctypes binding of the dgfas C ABI (include/dgfas.h).

Argument marshalling only: every step of the hot path runs in the sm_103a
kernels of libdgfas.so.  Device vectors are torch CUDA tensors (FP64,
contiguous); their data pointers and the current torch stream are passed to
the library.  The binding raises if the library is missing: there is no
fallback path.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgfas.so")

DGFAS_FP64, DGFAS_FP32, DGFAS_BF16 = 0, 1, 2
DGFAS_WAS, DGFAS_SCG = 0, 1
DGFAS_COARSE_DENSE, DGFAS_COARSE_SCG = 0, 1
DGFAS_P_INTERP, DGFAS_P_L2 = 0, 1
(DGFAS_OK, DGFAS_ERR_INVALID, DGFAS_ERR_OOM, DGFAS_ERR_CUDA, DGFAS_ERR_MESH,
 DGFAS_ERR_NOT_CONVERGED, DGFAS_ERR_DIVERGED, DGFAS_ERR_UNSUPPORTED) = 0, -1, -2, -3, -4, -5, -6, -7
ERRORS = {0: "ok", -1: "INVALID", -2: "OOM", -3: "CUDA", -4: "MESH", -5: "NOT_CONVERGED",
          -6: "DIVERGED", -7: "UNSUPPORTED"}


class DgfasError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} {detail}")


class dgfas_level(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("n_elem", ctypes.c_int),
                ("corners", ctypes.POINTER(ctypes.c_double)),
                ("nbr", ctypes.POINTER(ctypes.c_int)), ("nbr27", ctypes.POINTER(ctypes.c_int)),
                ("parent", ctypes.POINTER(ctypes.c_int)), ("octant", ctypes.POINTER(ctypes.c_int)),
                ("cls", ctypes.POINTER(ctypes.c_byte))]


class dgfas_mesh(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int), ("levels", ctypes.POINTER(dgfas_level)),
                ("nu", ctypes.c_double), ("kappa", ctypes.c_double)]


class dgfas_params(ctypes.Structure):
    _fields_ = [("mu_star", ctypes.c_double), ("delta", ctypes.c_double),
                ("s1", ctypes.c_int), ("s2", ctypes.c_int), ("sc", ctypes.c_int),
                ("precision", ctypes.c_int), ("smoother", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("coarse", ctypes.c_int),
                ("root_rtol", ctypes.c_double), ("root_steps", ctypes.c_int),
                ("projection", ctypes.c_int)]


class dgfas_info(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("r0", ctypes.c_double), ("r_final", ctypes.c_double),
                ("seconds", ctypes.c_double), ("history", ctypes.c_double * 128)]


SYMBOLS = ["dgfas_setup_levels", "dgfas_check_mesh", "dgfas_destroy", "dgfas_level_ndof", "dgfas_node_coords",
           "dgfas_assemble_rhs", "dgfas_apply_op", "dgfas_apply_op32", "dgfas_schwarz_smooth", "dgfas_fas_vcycle",
           "dgfas_solve", "dgfas_norm", "dgfas_set_surrogate", "dgfas_get_surrogate",
           "dgfas_use_graph", "dgfas_profile_sweep", "dgfas_profile_scg", "dgfas_scg_info", "dgfas_fma_peak", "dgfas_schwarz_correct_static", "dgfas_kernel_launches", "dgfas_mlp_param_count",
           "dgfas_mlp_forward", "dgfas_mlp_grad", "dgfas_mlp_inputs", "dgfas_mlp_train", "dgfas_learned_surrogate",
           "dgfas_assemble_rhs_level", "dgfas_set_level_rhs", "dgfas_composite_residual",
           "dgfas_get_level_solution", "dgfas_tc_selftest", "dgfas_tc_selftest_mn", "dgfas_tc_error", "dgfas_host_fd_variant", "dgfas_autotune", "dgfas_set_tuning",
           "dgfas_get_tuning", "dgfas_fmg", "dgfas_cmg", "dgfas_element_energy", "dgfas_strerror",
           "dgfas_last_error"]

_lib = None


def load():
    """Loads libdgfas.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} missing: run paper_2608_14123_b300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "dgfas_check_mesh": (I, [ctypes.POINTER(dgfas_mesh)]),
        "dgfas_setup_levels": (I, [ctypes.POINTER(dgfas_mesh), ctypes.POINTER(dgfas_params), P,
                                   ctypes.POINTER(P)]),
        "dgfas_destroy": (None, [P]),
        "dgfas_level_ndof": (LL, [P, I]),
        "dgfas_node_coords": (I, [P, I, P]),
        "dgfas_assemble_rhs": (I, [P, P, P, P]),
        "dgfas_apply_op": (I, [P, I, P, P, P]),
        "dgfas_apply_op32": (I, [P, I, P, P, P]),
        "dgfas_schwarz_smooth": (I, [P, I, P, P, I]),
        "dgfas_fas_vcycle": (I, [P, P, P, ctypes.POINTER(D)]),
        "dgfas_solve": (I, [P, P, P, D, I, ctypes.POINTER(dgfas_info)]),
        "dgfas_norm": (I, [P, I, P, ctypes.POINTER(D)]),
        "dgfas_set_surrogate": (I, [P, I, P]),
        "dgfas_get_surrogate": (I, [P, I, P]),
        "dgfas_use_graph": (I, [P, I]),
        "dgfas_host_fd_variant": (I, [I, D, D, I, P, P, P, ctypes.POINTER(I)]),
        "dgfas_profile_sweep": (I, [P, I, P, P, I, P]),
        "dgfas_profile_scg": (I, [P, I, P, P, I, P]),
        "dgfas_scg_info": (I, [P, P]),
        "dgfas_fma_peak": (I, [ctypes.POINTER(D), ctypes.POINTER(D)]),
        "dgfas_schwarz_correct_static": (I, [P, I, P, P]),
        "dgfas_kernel_launches": (LL, []),
        "dgfas_mlp_param_count": (I, []),
        "dgfas_mlp_forward": (I, [P, P, I, P, P]),
        "dgfas_mlp_inputs": (I, [P, I, P, P]),
        "dgfas_mlp_grad": (I, [P, P, P, I, P, P]),
        "dgfas_mlp_train": (I, [P, P, P, P, P, I, I, I, ctypes.c_float, ctypes.c_ulonglong, I, P, P]),
        "dgfas_learned_surrogate": (I, [P, I, P, D, ctypes.POINTER(I)]),
        "dgfas_assemble_rhs_level": (I, [P, I, P, P, P]),
        "dgfas_set_level_rhs": (I, [P, I, P]),
        "dgfas_composite_residual": (I, [P, P, P, ctypes.POINTER(D)]),
        "dgfas_get_level_solution": (I, [P, I, P]),
        "dgfas_tc_selftest": (I, [P, ctypes.POINTER(I)]),
        "dgfas_tc_error": (I, [P]),
        "dgfas_tc_selftest_mn": (I, [P, ctypes.POINTER(I)]),
        "dgfas_autotune": (I, [P, I, P, I, ctypes.POINTER(I)]),
        "dgfas_fmg": (I, [P, ctypes.POINTER(P), I, P]),
        "dgfas_cmg": (I, [P, ctypes.POINTER(P), I, P]),
        "dgfas_element_energy": (I, [P, I, P, P]),
        "dgfas_set_tuning": (I, [P, I, I, I]),
        "dgfas_get_tuning": (I, [P, I, I, ctypes.POINTER(I), P, I, ctypes.POINTER(I)]),
        "dgfas_strerror": (ctypes.c_char_p, [I]),
        "dgfas_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(code, where):
    if code != 0:
        raise DgfasError(code, where, load().dgfas_last_error().decode())
    return code


def _ptr(t, numel=None, dtype="float64"):
    """Device pointer of tensor t after checking what the kernels will assume:
    element type `dtype` (a torch dtype name), at least `numel` elements, a
    contiguous CUDA tensor.  A mismatch raises here, before any launch: a
    short or mistyped vector would otherwise be read or written out of bounds."""
    if t is None:
        return None
    if str(t.dtype) != "torch." + dtype:
        raise TypeError(f"expected a {dtype} tensor, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"tensor has {t.numel()} elements, the call needs {numel}")
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("device tensors must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Solver:
    """Owns one dgfas context: the hierarchy `levels` (root first, as produced by
    paper_2608_14123_b300.workloads) and the solver parameters."""

    def __init__(self, levels, mu_star, delta, s1=2, s2=2, sc=4, precision=DGFAS_FP64,
                 smoother=DGFAS_WAS, nu=1.0, kappa=0.0, max_cycles=50,
                 coarse=DGFAS_COARSE_DENSE, root_rtol=1e-3, root_steps=64,
                 projection=DGFAS_P_INTERP):
        lib = load()
        self._keep = []
        arr = (dgfas_level * len(levels))()
        for i, lv in enumerate(levels):
            ne = lv["nbr"].shape[0]
            corners = np.ascontiguousarray(lv["corners"], dtype=np.float64)
            nbr = np.ascontiguousarray(lv["nbr"], dtype=np.int32)
            nbr27 = np.ascontiguousarray(lv["nbr27"], dtype=np.int32)
            parent = np.ascontiguousarray(lv["parent"], dtype=np.int32)
            octant = np.ascontiguousarray(lv["octant"], dtype=np.int32)
            cls = np.ascontiguousarray(lv["cls"], dtype=np.int8)
            self._keep += [corners, nbr, nbr27, parent, octant, cls]
            arr[i] = dgfas_level(lv["p"], ne,
                                 corners.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 nbr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 nbr27.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 parent.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 octant.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 cls.ctypes.data_as(ctypes.POINTER(ctypes.c_byte)))
        mesh = dgfas_mesh(len(levels), arr, nu, kappa)
        prm = dgfas_params(mu_star, delta, s1, s2, sc, precision, smoother, max_cycles, coarse,
                           root_rtol, root_steps, projection)
        ctx = ctypes.c_void_p()
        _check(lib.dgfas_setup_levels(ctypes.byref(mesh), ctypes.byref(prm), _stream(),
                                      ctypes.byref(ctx)), "dgfas_setup_levels")
        self.ctx = ctx
        self.n_levels = len(levels)
        self.levels = levels
        self._keep = None

    def close(self):
        if getattr(self, "ctx", None):
            load().dgfas_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- ABI calls (same names, marshalling only)
    def ndof(self, level=-1):
        level = level % self.n_levels
        return int(load().dgfas_level_ndof(self.ctx, level))

    def n_elem(self, level=-1):
        return int(self.levels[level % self.n_levels]["nbr"].shape[0])

    def dgfas_node_coords(self, level, xyz):
        _check(load().dgfas_node_coords(self.ctx, level % self.n_levels,
                                            _ptr(xyz, 3 * self.ndof(level))), "node_coords")

    def dgfas_assemble_rhs(self, f, uD, b):
        n = self.ndof()
        _check(load().dgfas_assemble_rhs(self.ctx, _ptr(f, n), _ptr(uD, n), _ptr(b, n)), "assemble_rhs")

    def dgfas_apply_op(self, level, u, g, out):
        n = self.ndof(level)
        _check(load().dgfas_apply_op(self.ctx, level % self.n_levels, _ptr(u, n), _ptr(g, n),
                                     _ptr(out, n)),
               "apply_op")

    def dgfas_apply_op32(self, level, u, g, out):
        """FP32 operator: out = g - A u (g FP64) or A u (g None); u, out FP32."""
        n = self.ndof(level)
        _check(load().dgfas_apply_op32(self.ctx, level % self.n_levels, _ptr(u, n, "float32"),
                                       _ptr(g, n), _ptr(out, n, "float32")),
               "apply_op32")

    def dgfas_schwarz_smooth(self, level, u, g, n):
        nd = self.ndof(level)
        _check(load().dgfas_schwarz_smooth(self.ctx, level % self.n_levels, _ptr(u, nd), _ptr(g, nd),
                                           n),
               "schwarz_smooth")

    def dgfas_fas_vcycle(self, u, f, want_norm=True):
        r = ctypes.c_double(0.0)
        _check(load().dgfas_fas_vcycle(self.ctx, _ptr(u, self.ndof()), _ptr(f, self.ndof()),
                                       ctypes.byref(r) if want_norm else None), "fas_vcycle")
        return r.value

    def dgfas_solve(self, u, f, rtol=1e-10, max_cycles=50, raise_on_fail=True):
        info = dgfas_info()
        code = load().dgfas_solve(self.ctx, _ptr(u, self.ndof()), _ptr(f, self.ndof()), rtol, max_cycles, ctypes.byref(info))
        if raise_on_fail:
            _check(code, "solve")
        hist = [info.r0] + list(info.history[:min(info.cycles, 128)])
        return dict(code=code, cycles=info.cycles, r0=info.r0, r_final=info.r_final,
                    seconds=info.seconds, history=hist)

    def dgfas_norm(self, level, v):
        r = ctypes.c_double(0.0)
        _check(load().dgfas_norm(self.ctx, level % self.n_levels, _ptr(v, self.ndof(level)),
                                  ctypes.byref(r)), "norm")
        return r.value

    def dgfas_set_surrogate(self, level, g):
        _check(load().dgfas_set_surrogate(self.ctx, level % self.n_levels,
                                          _ptr(g, 4 * self.n_elem(level))), "set_surrogate")

    def dgfas_get_surrogate(self, level, g):
        _check(load().dgfas_get_surrogate(self.ctx, level % self.n_levels,
                                          _ptr(g, 4 * self.n_elem(level))), "get_surrogate")

    def dgfas_use_graph(self, enable):
        _check(load().dgfas_use_graph(self.ctx, 1 if enable else 0), "use_graph")

    def dgfas_profile_sweep(self, level, u, g, reps):
        ms = np.zeros(4)
        _check(load().dgfas_profile_sweep(self.ctx, level % self.n_levels, _ptr(u, self.ndof(level)),
                                          _ptr(g, self.ndof(level)), reps,
                                          ms.ctypes.data_as(ctypes.c_void_p)), "profile_sweep")
        return dict(residual_smoother=ms[0], fd=ms[1], combine=ms[2], residual_fp64=ms[3])

    def dgfas_profile_scg(self, level, u, g, reps):
        ms = np.zeros(6)
        _check(load().dgfas_profile_scg(self.ctx, level % self.n_levels, _ptr(u, self.ndof(level)),
                                        _ptr(g, self.ndof(level)), reps,
                                        ms.ctypes.data_as(ctypes.c_void_p)), "profile_scg")
        return dict(fd=ms[0], combine=ms[1], zr_dir=ms[2], apply_smoother=ms[3],
                    pq_update=ms[4], residual_fp64=ms[5])

    def dgfas_scg_info(self):
        """(|r|^2, steps, reached) of the last SCG block (synchronizes)."""
        out = np.zeros(3)
        _check(load().dgfas_scg_info(self.ctx, out.ctypes.data_as(ctypes.c_void_p)), "scg_info")
        return float(out[0]), int(out[1]), bool(out[2])

    def dgfas_fmg(self, f_levels, u_top, cycles_per_level=1):
        """Full multigrid startup (Alg. 4): u_top <- the FMG start value from the
        per-level right-hand sides f_levels (root first, device FP64)."""
        assert len(f_levels) == self.n_levels
        arr = (ctypes.c_void_p * self.n_levels)(*[_ptr(f, self.ndof(l)).value
                                                  for l, f in enumerate(f_levels)])
        _check(load().dgfas_fmg(self.ctx, arr, cycles_per_level, _ptr(u_top, self.ndof())), "fmg")

    def dgfas_cmg(self, f_levels, u_top, n_sc):
        """Cascadic startup (Alg. 3): u_top <- the CMG start value from the
        per-level right-hand sides f_levels (root first, device FP64), with
        n_sc smoothing steps on every intermediate level."""
        assert len(f_levels) == self.n_levels
        arr = (ctypes.c_void_p * self.n_levels)(*[_ptr(f, self.ndof(l)).value
                                                  for l, f in enumerate(f_levels)])
        _check(load().dgfas_cmg(self.ctx, arr, n_sc, _ptr(u_top, self.ndof())), "cmg")

    def dgfas_element_energy(self, level, eps, out):
        """out[e] = eps_e . (A eps)_e on `level` (element error indicators)."""
        _check(load().dgfas_element_energy(self.ctx, level % self.n_levels,
                                            _ptr(eps, self.ndof(level)),
                                            _ptr(out, self.n_elem(level))),
               "element_energy")

    TUNE_KERNELS = ("apply_fp64_elements_per_cta", "apply_smoother_elements_per_cta",
                    "fd_elements_per_cta", "fd_tensorcore_ctas_per_sm")

    def dgfas_autotune(self, reps=5):
        """Times the candidate launch shapes of the tunable kernels on every
        level and keeps the fastest; returns one dict per tuned (level, kernel)."""
        cap = 4 * 4 * self.n_levels
        rep = np.zeros((cap, 5))
        n = ctypes.c_int(0)
        _check(load().dgfas_autotune(self.ctx, reps, rep.ctypes.data_as(ctypes.c_void_p), cap,
                                     ctypes.byref(n)), "autotune")
        return [dict(level=int(r[0]), kernel=self.TUNE_KERNELS[int(r[1])], value=int(r[2]),
                     ms=float(r[3]), default_ms=float(r[4])) for r in rep[:n.value]]

    def dgfas_set_tuning(self, level, kernel, value):
        _check(load().dgfas_set_tuning(self.ctx, level % self.n_levels, kernel, value), "set_tuning")

    def dgfas_get_tuning(self, level, kernel):
        """(current value, candidate values) of `kernel` (0..3) on `level`."""
        v, n = ctypes.c_int(0), ctypes.c_int(0)
        cand = np.zeros(16, dtype=np.int32)
        _check(load().dgfas_get_tuning(self.ctx, level % self.n_levels, kernel, ctypes.byref(v),
                                       cand.ctypes.data_as(ctypes.c_void_p), 16, ctypes.byref(n)),
               "get_tuning")
        return v.value, [int(x) for x in cand[:n.value]]

    def dgfas_schwarz_correct_static(self, level, r, u):
        """u += weighted Schwarz correction of r, using the library's static
        scratch array (no device allocation in the call)."""
        _check(load().dgfas_schwarz_correct_static(self.ctx, level % self.n_levels,
                                                    _ptr(r, self.ndof(level)),
                                                    _ptr(u, self.ndof(level))),
               "schwarz_correct_static")

    def dgfas_learned_surrogate(self, level, params, max_log_scaling=2.5):
        """Surrogate coefficients of `level` from the MLP; returns the number of
        elements that kept their geometric coefficients."""
        nf = ctypes.c_int(0)
        _check(load().dgfas_learned_surrogate(self.ctx, level % self.n_levels,
                                              _ptr(params, load().dgfas_mlp_param_count(), "float32"),
                                              max_log_scaling, ctypes.byref(nf)), "learned_surrogate")
        return nf.value

    def dgfas_assemble_rhs_level(self, level, f, uD, b):
        n = self.ndof(level)
        _check(load().dgfas_assemble_rhs_level(self.ctx, level % self.n_levels, _ptr(f, n),
                                               _ptr(uD, n), _ptr(b, n)), "assemble_rhs_level")

    def dgfas_set_level_rhs(self, level, f):
        _check(load().dgfas_set_level_rhs(self.ctx, level, _ptr(f, self.ndof(level))), "set_level_rhs")

    def dgfas_composite_residual(self, u, f):
        r = ctypes.c_double(0.0)
        _check(load().dgfas_composite_residual(self.ctx, _ptr(u, self.ndof()), _ptr(f, self.ndof()),
                                               ctypes.byref(r)),
               "composite_residual")
        return r.value

    def dgfas_get_level_solution(self, level, u):
        _check(load().dgfas_get_level_solution(self.ctx, level, _ptr(u, self.ndof(level))), "get_level_solution")

    def dgfas_tc_error(self):
        return int(load().dgfas_tc_error(self.ctx))

    # ---- conveniences built from the calls above
    def node_coords(self, level=-1):
        import torch
        xyz = torch.empty((self.ndof(level), 3), dtype=torch.float64, device="cuda")
        self.dgfas_node_coords(level, xyz)
        return xyz


def dgfas_host_fd_variant(p, delta, mu_star, variant):
    """Host-side FD tables of one side variant: (S [n, n], lam [n], W [n])."""
    S = np.zeros(256)
    lam = np.zeros(16)
    W = np.zeros(16)
    n = ctypes.c_int(0)
    dp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(load().dgfas_host_fd_variant(p, delta, mu_star, variant, dp(S), dp(lam), dp(W),
                                        ctypes.byref(n)), "host_fd_variant")
    k = n.value
    return S[:k * k].reshape(k, k), lam[:k], W[:k]


def dgfas_fma_peak():
    """Measured FP64 and FP32 FMA throughput (TFLOP/s) of the current device."""
    a, b = ctypes.c_double(0), ctypes.c_double(0)
    _check(load().dgfas_fma_peak(ctypes.byref(a), ctypes.byref(b)), "fma_peak")
    return a.value, b.value


def dgfas_kernel_launches():
    """Kernels launched by the library so far in this process (graph nodes included)."""
    return int(load().dgfas_kernel_launches())


def dgfas_tc_selftest():
    """Runs the tcgen05 self-test; returns (D [128, 16], timed_out)."""
    out = np.zeros(128 * 16, dtype=np.float32)
    to = ctypes.c_int(0)
    _check(load().dgfas_tc_selftest(out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(to)),
           "tc_selftest")
    return out.reshape(128, 16), bool(to.value)
