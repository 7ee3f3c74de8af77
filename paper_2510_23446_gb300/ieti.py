"""ctypes binding of the C ABI declared in include/ieti.h (same names, marshalling only).

Device buffers may be passed as torch CUDA tensors (their data pointer is used);
host buffers as numpy arrays.  Nothing here computes: every step runs in
``libieti.so``, and importing this module raises if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libieti.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run paper_2510_23446_gb300.build.build()")
lib = C.CDLL(LIB_PATH)

IETI_MEM_HOST, IETI_MEM_DEVICE = 0, 1
PREC = {"fp64": 0, "mixed": 1}
PRECOND = {"none": 0, "dirichlet": 1, "dirichlet_mult": 2, "dirichlet_stiff": 3}
FACTOR = {"fp64": 0, "fp32": 1, "tf32x3": 2, "tf32": 3, "bf16x3": 4, "bf16": 5}
REFACTOR = {"every": 0, "step": 1, "never": 2}
COARSE = {"auto": 0, "dense": 1, "nd": 2}
ERRORS = {-1: "INVALID_ARG", -2: "NONCONFORMING", -3: "NOT_SPD", -4: "CG_NOT_CONVERGED", -5: "CUDA",
          -6: "OOM", -7: "NO_DEVICE", -8: "TOO_LARGE", -9: "TIMEOUT"}

_i32p = C.POINTER(C.c_int32)
_dp = C.POINTER(C.c_double)


class ieti_problem(C.Structure):
    _fields_ = [("n_patches", C.c_int32 * 3), ("n_el", _i32p * 3), ("degree", _i32p * 3),
                ("knots", _dp * 3), ("ctrl_pts", _dp), ("sigma_el", _dp), ("nu_el", _dp),
                ("dt", C.c_double), ("primal_mode", C.c_int32), ("reluctivity", _dp)]


class ieti_options(C.Structure):
    _fields_ = [("device", C.c_int32), ("precision", C.c_int32), ("precond", C.c_int32),
                ("cg_tol", C.c_double), ("cg_max_it", C.c_int32), ("outer_tol", C.c_double),
                ("max_sweeps", C.c_int32), ("pcg_mode", C.c_int32), ("host_threads", C.c_int32),
                ("cuda_stream", C.c_void_p), ("profile", C.c_int32), ("l2_persist", C.c_int32),
                ("factor", C.c_int32), ("refactor", C.c_int32), ("newton_tol", C.c_double),
                ("predictor", C.c_int32), ("autotune", C.c_int32), ("tune_cache", C.c_char_p),
                ("graph", C.c_int32), ("wait_limit", C.c_int32), ("coarse", C.c_int32),
                ("coarse_leaf", C.c_int32), ("factor_arena_mb", C.c_int32), ("coarse_top", C.c_int32),
                ("deflation", C.c_int32), ("coarse_ranks", C.c_int32)]


class ieti_coil(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("J0", "r_in", "r_out", "xc", "yc", "zc", "hz")]


class ieti_stats(C.Structure):
    _fields_ = [("cg_its", C.c_int32), ("sweeps", C.c_int32), ("rel_res", C.c_double),
                ("outer_res", C.c_double), ("t_step_ms", C.c_double), ("kernel_launches", C.c_int64),
                ("refactors", C.c_int32)]


class ieti_kernel_stat(C.Structure):
    _fields_ = [("launches", C.c_int64), ("total_ms", C.c_double), ("bytes", C.c_double)]


KERNEL_CLASSES = ["gemv_H", "gemv_Q", "gemv_P", "gemv_S", "gemv_Y", "tri", "spmv", "vec", "pcg"]


class ieti_info(C.Structure):
    _fields_ = [("n_dofs", C.c_int64), ("n_free", C.c_int64), ("n_lambda", C.c_int64),
                ("n_coarse", C.c_int64), ("sum_ni", C.c_int64), ("sum_nb", C.c_int64),
                ("sum_np", C.c_int64), ("max_n", C.c_int64), ("bytes_iter", C.c_int64),
                ("bytes_device", C.c_int64), ("t_setup_host_ms", C.c_double),
                ("t_setup_device_ms", C.c_double), ("kernel_launches_setup", C.c_int64),
                ("l2_window_bytes", C.c_int64), ("l2_hit_ratio", C.c_double), ("iter_operator_bytes", C.c_int64),
                ("t_factor_ms", C.c_double), ("tc_ms", C.c_double), ("tc_flops", C.c_double),
                ("tc_useful_flops", C.c_double), ("tc_launches", C.c_int64), ("factor_flops", C.c_double),
                ("nl_patches", C.c_int64), ("nl_elements", C.c_int64), ("refactors", C.c_int64),
                ("nl_coarse_block", C.c_int64), ("t_refactor_ms", C.c_double * 4),
                ("pcg_grid", C.c_int32), ("pcg_stages", C.c_int32), ("pcg_stage_bytes", C.c_int32),
                ("pcg_psi_partition", C.c_int32),
                ("pcg_sched_source", C.c_int32), ("tune_candidates", C.c_int32), ("tune_ms", C.c_double),
                ("tune_us_per_it", C.c_double * 2), ("step_graph", C.c_int32), ("coarse_mode", C.c_int32),
                ("coarse_nodes", C.c_int32), ("coarse_levels", C.c_int32), ("coarse_bytes", C.c_double),
                ("t_coarse_ms", C.c_double), ("factor_batches", C.c_int32), ("pcg_seg_weight", C.c_int32),
                ("coarse_flow", C.c_int32), ("deflation_dim", C.c_int32)]


_ctx = C.c_void_p
lib.ieti_setup.argtypes = [C.POINTER(ieti_problem), C.POINTER(ieti_options), C.POINTER(_ctx)]
lib.ieti_setup.restype = C.c_int
lib.ieti_setup_error.restype = C.c_char_p
lib.ieti_num_dofs.argtypes = [_ctx]
lib.ieti_num_dofs.restype = C.c_int64
lib.ieti_get_info.argtypes = [_ctx, C.POINTER(ieti_info)]
lib.ieti_load_vector.argtypes = [_ctx, C.POINTER(ieti_coil), C.c_void_p]
lib.ieti_dof_classes.argtypes = [_ctx, C.c_void_p, C.c_void_p]
lib.ieti_quad_points.argtypes = [_ctx, C.c_void_p, C.POINTER(C.c_int64)]
lib.ieti_load_vector_points.argtypes = [_ctx, C.c_void_p, C.c_void_p]
lib.ieti_patch_csr.argtypes = [_ctx, C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                               C.c_void_p, C.c_void_p, C.c_void_p]
lib.ieti_step.argtypes = [_ctx, C.c_void_p, C.c_int32, C.POINTER(ieti_stats)]
lib.ieti_solution.argtypes = [_ctx, C.c_void_p, C.c_int64, C.c_int32]
lib.ieti_set_state.argtypes = [_ctx, C.c_void_p, C.c_int64, C.c_int32]
lib.ieti_kernel_stats.argtypes = [_ctx, C.c_void_p, C.c_int32]
lib.ieti_coarse_tree.argtypes = [_ctx, C.POINTER(C.c_int32), C.POINTER(C.c_int64)] + [C.c_void_p] * 6
lib.ieti_pcg_phase_times.argtypes = [_ctx, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
lib.ieti_coarse_level_times.argtypes = [_ctx, C.c_void_p, C.c_int32, C.c_int32]
lib.ieti_shard_plan.argtypes = [_ctx, C.c_int32] + [C.c_void_p] * 4
lib.ieti_shard_coarse.argtypes = [_ctx, C.c_int32, C.c_void_p]
lib.ieti_multipliers.argtypes = [_ctx] + [C.c_void_p] * 4
lib.ieti_patch_blocks.argtypes = [_ctx] + [C.c_void_p] * 4
lib.ieti_potrf_batched.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p]
lib.ieti_potrf_batched_noalloc.argtypes = lib.ieti_potrf_batched.argtypes
lib.ieti_potrf_batched_f32.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_int32, C.c_void_p, C.c_void_p]
lib.ieti_last_error.argtypes = [_ctx]
lib.ieti_last_error.restype = C.c_char_p
lib.ieti_destroy.argtypes = [_ctx]
lib.ieti_destroy.restype = None

EXPORTED = ["ieti_setup", "ieti_setup_error", "ieti_num_dofs", "ieti_get_info", "ieti_load_vector",
            "ieti_dof_classes", "ieti_patch_csr", "ieti_step", "ieti_solution", "ieti_set_state",
            "ieti_last_error", "ieti_destroy", "ieti_kernel_stats", "ieti_pcg_phase_times",
            "ieti_potrf_batched", "ieti_potrf_batched_noalloc", "ieti_potrf_batched_f32",
            "ieti_quad_points", "ieti_load_vector_points", "ieti_coarse_tree", "ieti_coarse_level_times",
            "ieti_shard_plan", "ieti_shard_coarse", "ieti_multipliers", "ieti_patch_blocks"]


class IetiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _ptr(x):
    """Raw address of a numpy array (host) or a torch tensor (host or device)."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data, IETI_MEM_HOST
    dp = getattr(x, "data_ptr", None)
    if dp is not None:
        return dp(), (IETI_MEM_DEVICE if x.is_cuda else IETI_MEM_HOST)
    raise TypeError("expected a numpy array or a torch tensor")


class Solver:
    """One IETI-DP context (ieti_setup ... ieti_destroy)."""

    def __init__(self, P, n_el, degree, knots, ctrl, sigma_el, nu_el, dt, *, reluctivity=None, device=0,
                 precision="fp64", precond="dirichlet_stiff", cg_tol=1e-10, cg_max_it=5000,
                 outer_tol=1e-12, max_sweeps=None, pcg_mode=0, host_threads=0, stream=None, profile=0, l2_persist=2,
                 factor="fp64", refactor="every", newton_tol=0.0, predictor=0, autotune=0, tune_cache=None,
                 graph=1, wait_limit=0, coarse="auto", coarse_leaf=0, factor_arena_mb=0, coarse_top=0,
                 deflation=0, coarse_ranks=0):
        self._keep = []

        def arr(x, dt_):
            a = np.ascontiguousarray(np.asarray(x, dtype=dt_))
            self._keep.append(a)
            return a
        pr = ieti_problem()
        for d in range(3):
            pr.n_patches[d] = int(P[d])
            pr.n_el[d] = arr(n_el[d], np.int32).ctypes.data_as(_i32p)
            pr.degree[d] = arr(degree[d], np.int32).ctypes.data_as(_i32p)
            pr.knots[d] = arr(knots[d], np.float64).ctypes.data_as(_dp)
        pr.ctrl_pts = arr(ctrl, np.float64).ctypes.data_as(_dp)
        pr.sigma_el = arr(sigma_el, np.float64).ctypes.data_as(_dp)
        pr.nu_el = arr(nu_el, np.float64).ctypes.data_as(_dp)
        pr.dt = float(dt)
        pr.primal_mode = 0
        if reluctivity is not None:
            law = reluctivity
            if isinstance(law, dict):
                law = [law["nu0"], law["k1"], law["k2"], law["k3"]]
            pr.reluctivity = arr(law, np.float64).ctypes.data_as(_dp)
        op = ieti_options()
        op.device = int(device)
        op.precision = PREC[precision] if isinstance(precision, str) else int(precision)
        op.precond = PRECOND[precond] if isinstance(precond, str) else int(precond)
        op.cg_tol = float(cg_tol)
        op.cg_max_it = int(cg_max_it)
        op.outer_tol = float(outer_tol)
        if max_sweeps is None:
            max_sweeps = 1 if op.precision == 0 else 20
        op.max_sweeps = int(max_sweeps)
        op.pcg_mode = int(pcg_mode)
        op.host_threads = int(host_threads)
        op.cuda_stream = C.c_void_p(stream or 0)
        op.profile = int(profile)
        op.l2_persist = int(l2_persist)
        op.factor = FACTOR[factor] if isinstance(factor, str) else int(factor)
        op.refactor = REFACTOR[refactor] if isinstance(refactor, str) else int(refactor)
        op.newton_tol = float(newton_tol)
        op.predictor = int(predictor)
        op.autotune = int(autotune)
        op.graph = int(graph)
        op.wait_limit = int(wait_limit)
        op.coarse = COARSE[coarse] if isinstance(coarse, str) else int(coarse)
        op.coarse_leaf = int(coarse_leaf)
        op.coarse_top = int(coarse_top)
        op.deflation = int(deflation)
        op.coarse_ranks = int(coarse_ranks)
        op.factor_arena_mb = int(factor_arena_mb)
        if tune_cache is not None:
            op.tune_cache = os.fsencode(tune_cache)      # the structure keeps the bytes alive
        self.options = op
        self.ctx = _ctx()
        rc = lib.ieti_setup(C.byref(pr), C.byref(op), C.byref(self.ctx))
        self._keep = []
        if rc != 0:
            raise IetiError(rc, lib.ieti_setup_error().decode())
        self.n = int(lib.ieti_num_dofs(self.ctx))
        self._P = tuple(int(x) for x in P)

    @classmethod
    def from_problem(cls, prob, **kw):
        kw.setdefault("reluctivity", getattr(prob, "reluctivity", None))
        return cls(prob.P, prob.n_el, prob.degree, prob.knots, prob.ctrl, prob.sigma_el,
                   prob.nu_el, prob.dt, **kw)

    def _check(self, rc):
        if rc != 0:
            raise IetiError(rc, lib.ieti_last_error(self.ctx).decode())

    def info(self):
        inf = ieti_info()
        self._check(lib.ieti_get_info(self.ctx, C.byref(inf)))
        out = {k: getattr(inf, k) for k, _ in ieti_info._fields_}
        out["t_refactor_ms"] = list(out["t_refactor_ms"])
        out["tune_us_per_it"] = list(out["tune_us_per_it"])
        return out

    def quad_points(self):
        n = C.c_int64(0)
        self._check(lib.ieti_quad_points(self.ctx, None, C.byref(n)))
        xyz = np.zeros((n.value, 3))
        self._check(lib.ieti_quad_points(self.ctx, xyz.ctypes.data, C.byref(n)))
        return xyz

    def load_vector_points(self, J):
        J = np.ascontiguousarray(J, dtype=np.float64)
        out = np.zeros(self.n)
        self._check(lib.ieti_load_vector_points(self.ctx, J.ctypes.data, out.ctypes.data))
        return out

    def load_vector(self, coil):
        c = ieti_coil(**{k: float(coil[k]) for k, _ in ieti_coil._fields_})
        out = np.zeros(self.n)
        self._check(lib.ieti_load_vector(self.ctx, C.byref(c), out.ctypes.data))
        return out

    def dof_classes(self):
        cls = np.zeros(self.n, dtype=np.int8)
        tree = np.zeros(self.n, dtype=np.int8)
        self._check(lib.ieti_dof_classes(self.ctx, cls.ctypes.data, tree.ctypes.data))
        return cls, tree

    def patch_csr(self, s, which):
        n = C.c_int32()
        nnz = C.c_int64()
        self._check(lib.ieti_patch_csr(self.ctx, s, which, C.byref(n), C.byref(nnz), None, None, None))
        ptr = np.zeros(n.value + 1, dtype=np.int32)
        col = np.zeros(nnz.value, dtype=np.int32)
        val = np.zeros(nnz.value)
        self._check(lib.ieti_patch_csr(self.ctx, s, which, None, None, ptr.ctypes.data,
                                       col.ctypes.data, val.ctypes.data))
        return ptr, col, val

    def coarse_tree(self):
        """ieti_coarse_tree: the nested-dissection tree of the coarse problem."""
        nn = C.c_int32()
        ns = C.c_int64()
        self._check(lib.ieti_coarse_tree(self.ctx, C.byref(nn), C.byref(ns), None, None, None, None, None, None))
        elim = np.zeros(self.n, dtype=np.int32)
        k0 = np.zeros(nn.value, dtype=np.int32)
        nk = np.zeros(nn.value, dtype=np.int32)
        parent = np.zeros(nn.value, dtype=np.int32)
        s_off = np.zeros(nn.value + 1, dtype=np.int64)
        s_idx = np.zeros(max(ns.value, 1), dtype=np.int32)
        self._check(lib.ieti_coarse_tree(self.ctx, C.byref(nn), C.byref(ns), elim.ctypes.data, k0.ctypes.data,
                                         nk.ctypes.data, parent.ctypes.data, s_off.ctypes.data, s_idx.ctypes.data))
        return dict(elim_pos=elim, k0=k0, nk=nk, parent=parent, s_off=s_off, s_idx=s_idx[:ns.value])

    def kernel_stats(self, reset=False):
        arr = (ieti_kernel_stat * len(KERNEL_CLASSES))()
        self._check(lib.ieti_kernel_stats(self.ctx, C.cast(arr, C.c_void_p), int(reset)))
        return {name: {"launches": arr[i].launches, "total_ms": arr[i].total_ms, "bytes": arr[i].bytes}
                for i, name in enumerate(KERNEL_CLASSES)}

    def pcg_phase_times(self, reset=False):
        work = np.zeros(6)
        wait = np.zeros(6)
        sub = np.zeros(12)
        self._check(lib.ieti_pcg_phase_times(self.ctx, work.ctypes.data, wait.ctypes.data, sub.ctypes.data,
                                             int(reset)))
        return {"work_us": work.tolist(), "wait_us": wait.tolist(), "sub_us": sub.reshape(4, 3).tolist()}

    def shard_plan(self, n_ranks):
        """ieti_shard_plan: rank of every patch, owner and peer rank of every multiplier,
        owner of every coarse unknown."""
        inf = self.info()
        npat = int(np.prod(self._P))
        rop = np.zeros(npat, dtype=np.int32)
        own = np.zeros(inf["n_lambda"], dtype=np.int32)
        peer = np.zeros(inf["n_lambda"], dtype=np.int32)
        cown = np.zeros(max(inf["n_coarse"], 1), dtype=np.int32)
        self._check(lib.ieti_shard_plan(self.ctx, int(n_ranks), rop.ctypes.data, own.ctypes.data, peer.ctypes.data,
                                        cown.ctypes.data))
        return dict(rank_of_patch=rop, lam_owner=own, lam_peer=peer, coarse_owner=cown[:inf["n_coarse"]])

    def shard_coarse(self, n_ranks):
        """ieti_shard_coarse: the rank computing every node of the coarse tree (-1: shared)."""
        n = len(self.coarse_tree()["k0"])
        out = np.zeros(max(n, 1), dtype=np.int32)
        self._check(lib.ieti_shard_coarse(self.ctx, int(n_ranks), out.ctypes.data))
        return out[:n]

    def multipliers(self):
        m = self.info()["n_lambda"]
        out = [np.zeros(m, dtype=np.int32) for _ in range(4)]
        self._check(lib.ieti_multipliers(self.ctx, *[a.ctypes.data for a in out]))
        return dict(zip(("s", "pos_s", "t", "pos_t"), out))

    def patch_blocks(self):
        npat = int(np.prod(self._P))
        ni, nb, np_ = (np.zeros(npat, dtype=np.int32) for _ in range(3))
        self._check(lib.ieti_patch_blocks(self.ctx, ni.ctypes.data, nb.ctypes.data, np_.ctypes.data, None))
        cc = np.zeros(max(int(np_.sum()), 1), dtype=np.int32)
        self._check(lib.ieti_patch_blocks(self.ctx, None, None, None, cc.ctypes.data))
        return dict(ni=ni, nb=nb, np=np_, coarse_of_copy=cc[:int(np_.sum())])

    def coarse_level_times(self, reset=False):
        """Per level of the nested-dissection coarse solve: [staging, first chunk, rows,
        barrier wait] in microseconds (CTA 0, mean over the traced iterations)."""
        n = 4 * 24
        us = np.zeros(n)
        self._check(lib.ieti_coarse_level_times(self.ctx, us.ctypes.data, n, int(reset)))
        return us.reshape(24, 4)[:min(24, self.info()["coarse_levels"])].tolist()

    def step(self, j, raise_on_error=True):
        p, mem = _ptr(j)
        st = ieti_stats()
        rc = lib.ieti_step(self.ctx, C.c_void_p(p), mem, C.byref(st))
        if rc != 0 and raise_on_error:
            self._check(rc)
        return {k: getattr(st, k) for k, _ in ieti_stats._fields_} | {"rc": rc}

    def solution(self, out=None):
        if out is None:
            out = np.zeros(self.n)
        p, mem = _ptr(out)
        self._check(lib.ieti_solution(self.ctx, C.c_void_p(p), self.n, mem))
        return out

    def set_state(self, a):
        p, mem = _ptr(a)
        self._check(lib.ieti_set_state(self.ctx, C.c_void_p(p), self.n, mem))

    def close(self):
        if self.ctx:
            lib.ieti_destroy(self.ctx)
            self.ctx = _ctx()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def potrf_batched(base, offsets, n, n_pivots, stream=0, noalloc=False):
    """ieti_potrf_batched (or, with noalloc=True, ieti_potrf_batched_noalloc, which
    allocates no device memory) on a device buffer `base` (torch CUDA float64 tensor).

    Returns the per-matrix status array (0 = all pivots positive)."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    nn = np.ascontiguousarray(np.asarray(n, dtype=np.int32))
    kp = np.ascontiguousarray(np.asarray(n_pivots, dtype=np.int32))
    st = np.zeros(len(nn), dtype=np.int32)
    p, mem = _ptr(base)
    if mem != IETI_MEM_DEVICE:
        raise TypeError("base must be a CUDA tensor")
    fn = lib.ieti_potrf_batched_noalloc if noalloc else lib.ieti_potrf_batched
    rc = fn(len(nn), C.c_void_p(p), off.ctypes.data, nn.ctypes.data, kp.ctypes.data, st.ctypes.data,
            C.c_void_p(stream or 0))
    if rc != 0:
        raise IetiError(rc, lib.ieti_setup_error().decode())
    return st


def potrf_batched_f32(base, offsets, n, ld, n_pivots, factor="tf32x3", stream=0):
    """ieti_potrf_batched_f32 on a device buffer `base` (torch CUDA float32 tensor):
    the FP32 batched partial Cholesky with SIMT ("fp32") or tensor-core ("tf32x3",
    "tf32") trailing updates.  Returns the per-matrix status array."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    nn = np.ascontiguousarray(np.asarray(n, dtype=np.int32))
    ldv = np.ascontiguousarray(np.asarray(ld, dtype=np.int32))
    kp = np.ascontiguousarray(np.asarray(n_pivots, dtype=np.int32))
    st = np.zeros(len(nn), dtype=np.int32)
    p, mem = _ptr(base)
    if mem != IETI_MEM_DEVICE:
        raise TypeError("base must be a CUDA tensor")
    f = FACTOR[factor] if isinstance(factor, str) else int(factor)
    rc = lib.ieti_potrf_batched_f32(len(nn), C.c_void_p(p), off.ctypes.data, nn.ctypes.data, ldv.ctypes.data,
                                    kp.ctypes.data, f, st.ctypes.data, C.c_void_p(stream or 0))
    if rc != 0:
        raise IetiError(rc, lib.ieti_setup_error().decode())
    return st
