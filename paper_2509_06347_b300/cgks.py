"""Thin Python binding of the CGKS C ABI (include/cgks.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
Device arrays are torch CUDA tensors (passed by data_ptr); host arrays are
numpy arrays.  Importing works without a GPU; loading the library requires the
built libcgks.so and raises if it is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcgks.so")

CGKS_OK = 0
ERRORS = {-1: "CGKS_ERR_ARG", -2: "CGKS_ERR_MESH", -3: "CGKS_ERR_CUDA", -4: "CGKS_ERR_DIVERGED",
          -5: "CGKS_ERR_NONPOSITIVE", -6: "CGKS_ERR_TIMEOUT", -7: "CGKS_ERR_STATE"}
PLAIN_FP64, MIXED, LEARNED = 0, 1, 2
TAG_WALL, TAG_FARFIELD, TAG_NOSLIP_WALL, TAG_FARFIELD_RIEMANN = 1, 2, 3, 4

# every entry point declared in include/cgks.h
EXPORTS = ["cgks_default_config", "cgks_create", "cgks_destroy", "cgks_last_error", "cgks_upload_mesh",
           "cgks_upload_mesh_mixed",
           "cgks_upload_hierarchy", "cgks_agglomerate", "cgks_mesh_info", "cgks_get_hierarchy", "cgks_get_coloring", "cgks_set_freestream",
           "cgks_init_state", "cgks_get_state", "cgks_set_state", "cgks_residual", "cgks_reconstruct",
           "cgks_lusgs", "cgks_smooth", "cgks_vcycle", "cgks_residual_norms", "cgks_counters",
           "cgks_gks_points", "cgks_kfvs_points", "cgks_run_stage", "cgks_launch_count",
           "cgks_vcycle_launch", "cgks_dword_selftest", "cgks_special_selftest", "cgks_fma_probe", "cgks_set_groups", "cgks_vcycle_groups",
           "cgks_autotune", "cgks_residual_coarse_noalloc", "cgks_mlp_set_params", "cgks_mlp_get_params",
           "cgks_mlp_forward", "cgks_mlp_select", "cgks_mlp_grad", "cgks_mlp_dataset_append", "cgks_mlp_dataset_size",
           "cgks_mlp_dataset_clear", "cgks_mlp_train", "cgks_mlp_collect", "cgks_mlp_features", "cgks_learned_stats",
           "cgks_synchronize"]


# the per-cell network: inputs and parameter count
N_IN = 76
N_PARAMS = 64 * N_IN + 64 + 64 * 64 + 64 + 4 * 64 + 4  # 9,348


class CgksError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl_imp", C.c_double), ("cfl_exp", C.c_double),
                ("tau_c1", C.c_double), ("tau_c2", C.c_double), ("weno_gamma_high", C.c_double),
                ("weno_eps", C.c_double), ("r_safety", C.c_double), ("n_sweep_coarse", C.c_int),
                ("n_pre", C.c_int), ("n_post", C.c_int), ("check_every", C.c_int), ("tol", C.c_double),
                ("diverge_factor", C.c_double), ("fine_smoother", C.c_int), ("df_relax", C.c_int),
                ("df_prolong", C.c_int), ("df_gate", C.c_double), ("learned_judge_every", C.c_int),
                ("learned_max_error", C.c_double), ("flux_precision", C.c_int),
                ("relax_beta", C.c_double), ("mu", C.c_double), ("slope_relax", C.c_double),
                ("alpha_relax", C.c_double), ("learned_scale", C.c_int),
                ("coarse_cluster_max_cells", C.c_int)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libcgks.so (raises FileNotFoundError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"CGKS CUDA library not built: {path} "
                                "(run python -m paper_2509_06347_b300.build)")
    L = C.CDLL(path)
    P, I, I64, D = C.c_void_p, C.c_int, C.c_int64, C.c_double
    sig = {
        "cgks_default_config": [C.POINTER(Config)],
        "cgks_create": [C.POINTER(C.c_void_p), C.POINTER(Config), P],
        "cgks_destroy": [P],
        "cgks_upload_mesh": [P, I, I, I64, P, P, I64, P, P],
        "cgks_upload_mesh_mixed": [P, I, I64, P, P, P, P, I64, P, P, P],
        "cgks_upload_hierarchy": [P, I, I, P],
        "cgks_mesh_info": [P, I, P, P],
        "cgks_agglomerate": [P, I, I64, P, P, I64, P, P, I, I, D, P, P],
        "cgks_dword_selftest": [P, I64, P, P, P],
        "cgks_special_selftest": [P, I64, P, P],
        "cgks_mlp_features": [P, I, P],
        "cgks_get_coloring": [P, I, I, P],
        "cgks_get_hierarchy": [P, I, I, P, P],
        "cgks_set_freestream": [P, I, P],
        "cgks_init_state": [P, I, P, P, I],
        "cgks_get_state": [P, I, P, P, P, I],
        "cgks_set_state": [P, I, P, P, P, I],
        "cgks_residual": [P, I, I, P, P, P, P, I],
        "cgks_reconstruct": [P, I, P, P, P, I],
        "cgks_lusgs": [P, I, I, I, P, P, P, P, P, P, I],
        "cgks_smooth": [P, I, I, I],
        "cgks_vcycle": [P, P, I, I, I, P, P],
        "cgks_residual_norms": [P, I, I, P],
        "cgks_counters": [P, I, P],
        "cgks_gks_points": [P, I, I64, P, P, P, P, P, P, P, P],
        "cgks_kfvs_points": [P, I, I64, P, P, P],
        "cgks_run_stage": [P, I, I],
        "cgks_vcycle_launch": [P, P, I, I, I],
        "cgks_fma_probe": [P, I, P],
        "cgks_set_groups": [P, I, I, P, P],
        "cgks_vcycle_groups": [P, I, I, I, P, P, P],
        "cgks_autotune": [P, I, P],
        "cgks_residual_coarse_noalloc": [P, I, I, P, P],
        "cgks_mlp_set_params": [P, P],
        "cgks_mlp_get_params": [P, P],
        "cgks_mlp_forward": [P, I64, P, P],
        "cgks_mlp_select": [P, I],
        "cgks_mlp_grad": [P, I64, P, P, P, P],
        "cgks_mlp_dataset_append": [P, I64, P, P],
        "cgks_mlp_dataset_size": [P, P],
        "cgks_mlp_dataset_clear": [P],
        "cgks_mlp_train": [P, I, I, C.c_double, C.c_uint64, P],
        "cgks_mlp_collect": [P, I, I, I],
        "cgks_learned_stats": [P, I, P],
        "cgks_launch_count": [P, I, I, P],
        "cgks_synchronize": [P],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.cgks_last_error.argtypes = [P]
    L.cgks_last_error.restype = C.c_char_p
    _lib = L
    return L


def default_config(**over) -> Config:
    cfg = Config()
    load_library().cgks_default_config(C.byref(cfg))
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg


def _ptr(a):
    """Address of a torch tensor (device or host) or numpy array; None -> NULL."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _is_dev(a):
    return hasattr(a, "is_cuda") and a.is_cuda


class Context:
    """One cgks_t handle bound to a CUDA stream (0 = library-private stream)."""

    def __init__(self, config: Config | None = None, stream: int = 0, **over):
        L = load_library()
        self._L = L
        cfg = config if config is not None else default_config(**over)
        self.config = cfg
        h = C.c_void_p()
        rc = L.cgks_create(C.byref(h), C.byref(cfg), C.c_void_p(stream) if stream else None)
        if rc != CGKS_OK:
            raise CgksError(rc, "cgks_create failed")
        self.h = h
        self.meshes = {}

    def close(self):
        if getattr(self, "h", None):
            self._L.cgks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != CGKS_OK:
            raise CgksError(rc, self._L.cgks_last_error(self.h).decode())
        return rc

    # ---- mesh ----------------------------------------------------------------
    def cgks_upload_mesh(self, mesh_id: int, mesh: dict):
        cn = np.ascontiguousarray(mesh["cell_nodes"], np.int32)
        cx = np.ascontiguousarray(mesh["cell_xyz"], np.float64)
        bn = np.ascontiguousarray(mesh["bface_nodes"], np.int32)
        bt = np.ascontiguousarray(mesh["bface_tag"], np.int32)
        self._check(self._L.cgks_upload_mesh(self.h, mesh_id, int(mesh["dim"]), cn.shape[0], _ptr(cn), _ptr(cx),
                                              bt.size, _ptr(bn) if bt.size else None, _ptr(bt) if bt.size else None))
        self.meshes[mesh_id] = dict(dim=int(mesh["dim"]), n=cn.shape[0])

    def cgks_upload_mesh_mixed(self, mesh_id: int, mesh: dict):
        """Mixed-element 3-D mesh (cell types by node count; see the header)."""
        ct = np.ascontiguousarray(mesh["cell_type"], np.int32)
        co = np.ascontiguousarray(mesh["cell_node_off"], np.int64)
        cn = np.ascontiguousarray(mesh["cell_nodes"], np.int32)
        cx = np.ascontiguousarray(mesh["cell_xyz"], np.float64)
        bo = np.ascontiguousarray(mesh["bface_node_off"], np.int64)
        bn = np.ascontiguousarray(mesh["bface_nodes"], np.int32)
        bt = np.ascontiguousarray(mesh["bface_tag"], np.int32)
        self._check(self._L.cgks_upload_mesh_mixed(self.h, mesh_id, ct.size, _ptr(ct), _ptr(co), _ptr(cn), _ptr(cx),
                                                    bt.size, _ptr(bo) if bt.size else None,
                                                    _ptr(bn) if bt.size else None, _ptr(bt) if bt.size else None))
        self.meshes[mesh_id] = dict(dim=3, n=ct.size)

    def cgks_upload_hierarchy(self, mesh_id: int, parents):
        arrs = [np.ascontiguousarray(p, np.int32) for p in parents]
        ptrs = (C.c_void_p * max(1, len(arrs)))(*[a.ctypes.data for a in arrs])
        self._check(self._L.cgks_upload_hierarchy(self.h, mesh_id, len(arrs) + 1, ptrs))

    def cgks_agglomerate(self, mesh: dict, n_levels: int = 3, passes: int = 3, min_skew: float = 0.1):
        """Parent arrays of an agglomerated hierarchy (list of n_levels - 1 int32
        arrays, original numbering), for cgks_upload_hierarchy.  Three pairwise
        passes per level give about 3.5:1 in 2D and 3:1 in 3D on the first level."""
        dim = int(mesh["dim"])
        cn = np.ascontiguousarray(mesh["cell_nodes"], np.int32)
        cx = np.ascontiguousarray(mesh["cell_xyz"], np.float64)
        bn = np.ascontiguousarray(mesh["bface_nodes"], np.int32)
        bt = np.ascontiguousarray(mesh["bface_tag"], np.int32)
        n = cn.shape[0]
        par = np.zeros(max(1, (n_levels - 1) * n), np.int32)
        sizes = np.zeros(n_levels, np.int64)
        self._check(self._L.cgks_agglomerate(self.h, dim, n, _ptr(cn), _ptr(cx), bt.size,
                                             _ptr(bn) if bt.size else None, _ptr(bt) if bt.size else None,
                                             n_levels, passes, float(min_skew), _ptr(par), _ptr(sizes)))
        return [par[(l - 1) * n:(l - 1) * n + sizes[l - 1]].copy() for l in range(1, n_levels)]

    def cgks_mesh_info(self, mesh_id: int):
        nl = C.c_int()
        out = np.zeros(32, np.int64)
        self._check(self._L.cgks_mesh_info(self.h, mesh_id, C.byref(nl), _ptr(out)))
        return [dict(cells=int(out[4 * l]), colors=int(out[4 * l + 1]), faces=int(out[4 * l + 2]),
                     bfaces=int(out[4 * l + 3])) for l in range(nl.value)]

    def cgks_get_hierarchy(self, mesh_id: int, level: int, n: int, with_parent: bool = True):
        """(order, parent): the stored (colour-major) order of a level as original
        ids, and each cell's agglomerate on the next level (None on the coarsest)."""
        order = np.zeros(n, np.int32)
        parent = np.zeros(n, np.int32) if with_parent else None
        self._check(self._L.cgks_get_hierarchy(self.h, mesh_id, level, _ptr(order), _ptr(parent)))
        return order, parent

    def cgks_get_coloring(self, mesh_id: int, level: int, n: int):
        out = np.zeros(n, np.int32)
        self._check(self._L.cgks_get_coloring(self.h, mesh_id, level, _ptr(out)))
        return out

    def cgks_set_freestream(self, mesh_id: int, w):
        w = np.ascontiguousarray(w, np.float64)
        self._check(self._L.cgks_set_freestream(self.h, mesh_id, _ptr(w)))

    # ---- state -----------------------------------------------------------------
    def cgks_init_state(self, mesh_id: int, W, grad=None):
        dev = _is_dev(W)
        if not dev:
            W = np.ascontiguousarray(W, np.float64)
            grad = None if grad is None else np.ascontiguousarray(grad, np.float64)
        self._check(self._L.cgks_init_state(self.h, mesh_id, _ptr(W), _ptr(grad), int(dev)))

    def cgks_set_state(self, mesh_id: int, W=None, grad=None, alpha=None):
        arrs = [W, grad, alpha]
        dev = any(_is_dev(a) for a in arrs if a is not None)
        if not dev:
            arrs = [None if a is None else np.ascontiguousarray(a, np.float64) for a in arrs]
        self._check(self._L.cgks_set_state(self.h, mesh_id, *[_ptr(a) for a in arrs], int(dev)))

    def cgks_get_state(self, mesh_id: int, W=None, grad=None, alpha=None):
        """Fills the given arrays (all torch CUDA tensors, or all numpy arrays)."""
        arrs = [W, grad, alpha]
        dev = any(_is_dev(a) for a in arrs if a is not None)
        self._check(self._L.cgks_get_state(self.h, mesh_id, *[_ptr(a) for a in arrs], int(dev)))
        return W, grad, alpha

    def cgks_residual(self, mesh_id: int, level: int = 0, W_in=None, R=None, grad_new=None, alpha=None):
        arrs = [W_in, R, grad_new, alpha]
        dev = any(_is_dev(a) for a in arrs if a is not None)
        self._check(self._L.cgks_residual(self.h, mesh_id, level, *[_ptr(a) for a in arrs], int(dev)))
        return R, grad_new, alpha

    def cgks_reconstruct(self, mesh_id: int, coef=None, dt_exp=None, dt_imp=None):
        arrs = [coef, dt_exp, dt_imp]
        dev = any(_is_dev(a) for a in arrs if a is not None)
        self._check(self._L.cgks_reconstruct(self.h, mesh_id, *[_ptr(a) for a in arrs], int(dev)))
        return coef, dt_exp, dt_imp

    def cgks_lusgs(self, mesh_id: int, level: int, mode: int, W, rhs, alpha, dt_exp, dt_imp, dW=None):
        arrs = [W, rhs, alpha, dt_exp, dt_imp, dW]
        dev = any(_is_dev(a) for a in arrs if a is not None)
        self._check(self._L.cgks_lusgs(self.h, mesh_id, level, mode, *[_ptr(a) for a in arrs], int(dev)))
        return W, dW

    def cgks_smooth(self, mesh_id: int, level: int, n_sweeps: int):
        self._check(self._L.cgks_smooth(self.h, mesh_id, level, n_sweeps))

    def cgks_vcycle(self, mesh_ids, n_cycles: int, mode: int = PLAIN_FP64, norms=None, cycles_done=None,
                    check: bool = True):
        ids = np.ascontiguousarray(mesh_ids, np.int32)
        rc = self._L.cgks_vcycle(self.h, _ptr(ids), ids.size, n_cycles, mode, _ptr(norms), _ptr(cycles_done))
        if check:
            self._check(rc)
        return rc

    def cgks_residual_norms(self, mesh_id: int, level: int = 0):
        nv = self.meshes[mesh_id]["dim"] + 2
        out = np.zeros((nv, 2))
        self._check(self._L.cgks_residual_norms(self.h, mesh_id, level, _ptr(out)))
        return out

    def cgks_counters(self, mesh_id: int):
        out = np.zeros(4, np.uint64)
        self._check(self._L.cgks_counters(self.h, mesh_id, _ptr(out)))
        return out

    def cgks_gks_points(self, dim, Wl, Gl, Wr, Gr, dt, F, Wt, alpha):
        self._check(self._L.cgks_gks_points(self.h, dim, Wl.shape[0], *[_ptr(a) for a in (Wl, Gl, Wr, Gr, dt, F, Wt,
                                                                                          alpha)]))

    def cgks_kfvs_points(self, dim, Wl, Wr, F):
        self._check(self._L.cgks_kfvs_points(self.h, dim, Wl.shape[0], _ptr(Wl), _ptr(Wr), _ptr(F)))

    def cgks_vcycle_launch(self, mesh_ids, n_cycles: int, mode: int = PLAIN_FP64):
        ids = np.ascontiguousarray(mesh_ids, np.int32)
        self._check(self._L.cgks_vcycle_launch(self.h, _ptr(ids), ids.size, n_cycles, mode))

    def cgks_dword_selftest(self, a, b):
        a = np.ascontiguousarray(a, np.float64)
        b = np.ascontiguousarray(b, np.float64)
        out = np.zeros((a.size, 7))
        self._check(self._L.cgks_dword_selftest(self.h, a.size, _ptr(a), _ptr(b), _ptr(out)))
        return out

    def cgks_special_selftest(self, x):
        x = np.ascontiguousarray(x, np.float64)
        out = np.zeros((x.size, 5))
        self._check(self._L.cgks_special_selftest(self.h, x.size, _ptr(x) if x.size else None,
                                                  _ptr(out) if x.size else None))
        return out

    def cgks_fma_probe(self, precision: int = 0) -> float:
        out = C.c_double()
        self._check(self._L.cgks_fma_probe(self.h, precision, C.byref(out)))
        return out.value

    def cgks_set_groups(self, mesh_id: int, group_of_cell, winf):
        g = np.ascontiguousarray(group_of_cell, np.int32)
        w = np.ascontiguousarray(winf, np.float64)
        self._check(self._L.cgks_set_groups(self.h, mesh_id, w.shape[0], _ptr(g), _ptr(w)))
        self.meshes[mesh_id]["groups"] = w.shape[0]

    def cgks_vcycle_groups(self, mesh_id: int, n_cycles: int, mode: int = PLAIN_FP64, norms=None, check=True):
        G = self.meshes[mesh_id]["groups"]
        conv = np.zeros(G, np.int32)
        done = C.c_int()
        rc = self._L.cgks_vcycle_groups(self.h, mesh_id, n_cycles, mode, _ptr(norms), _ptr(conv), C.byref(done))
        if check:
            self._check(rc)
        return conv, done.value, rc

    def cgks_autotune(self, mesh_id: int):
        out = np.zeros(7, np.int32)
        self._check(self._L.cgks_autotune(self.h, mesh_id, _ptr(out)))
        return out

    def cgks_residual_coarse_noalloc(self, mesh_id: int, level: int, W_dev, R_dev, check: bool = True):
        """Coarse KFVS residual into a caller device buffer without any allocation."""
        rc = self._L.cgks_residual_coarse_noalloc(self.h, mesh_id, level, _ptr(W_dev), _ptr(R_dev))
        if check:
            self._check(rc)
        return rc

    # ---- learned correction -------------------------------------------------------
    def cgks_mlp_set_params(self, theta):
        t = np.ascontiguousarray(theta, np.float32)
        self._check(self._L.cgks_mlp_set_params(self.h, _ptr(t)))

    def cgks_mlp_get_params(self):
        out = np.zeros(N_PARAMS, np.float32)
        self._check(self._L.cgks_mlp_get_params(self.h, _ptr(out)))
        return out

    def cgks_mlp_select(self, impl: int):
        """Network forward implementation: 0 tcgen05 (tensor memory), 1 mma.sync."""
        self._check(self._L.cgks_mlp_select(self.h, int(impl)))

    def cgks_mlp_forward(self, X_bf16_dev, P_dev):
        self._check(self._L.cgks_mlp_forward(self.h, X_bf16_dev.shape[0], _ptr(X_bf16_dev), _ptr(P_dev)))

    def cgks_mlp_grad(self, X_bf16_dev, Y_dev, grad_dev):
        loss = C.c_float()
        self._check(self._L.cgks_mlp_grad(self.h, X_bf16_dev.shape[0], _ptr(X_bf16_dev), _ptr(Y_dev),
                                          _ptr(grad_dev), C.byref(loss)))
        return loss.value

    def cgks_mlp_dataset_append(self, X, Y):
        self._check(self._L.cgks_mlp_dataset_append(self.h, X.shape[0], _ptr(X), _ptr(Y)))

    def cgks_mlp_dataset_size(self):
        n = C.c_int64()
        self._check(self._L.cgks_mlp_dataset_size(self.h, C.byref(n)))
        return n.value

    def cgks_mlp_dataset_clear(self):
        self._check(self._L.cgks_mlp_dataset_clear(self.h))

    def cgks_mlp_train(self, n_steps: int, batch: int, lr: float, seed: int = 0):
        losses = np.zeros(max(1, n_steps), np.float32)
        self._check(self._L.cgks_mlp_train(self.h, n_steps, batch, lr, seed, _ptr(losses)))
        return losses[:n_steps]

    def cgks_mlp_collect(self, mesh_id: int, n_cycles: int, mode: int = PLAIN_FP64):
        self._check(self._L.cgks_mlp_collect(self.h, mesh_id, n_cycles, mode))

    def cgks_mlp_features(self, mesh_id: int):
        """Network inputs [n, 76] of the current state, as float32."""
        n = self.meshes[mesh_id]["n"]
        bits = np.zeros((n, N_IN), np.uint16)
        self._check(self._L.cgks_mlp_features(self.h, mesh_id, _ptr(bits)))
        return (bits.astype(np.uint32) << 16).view(np.float32)

    def cgks_learned_stats(self, mesh_id: int):
        out = np.zeros(10)
        self._check(self._L.cgks_learned_stats(self.h, mesh_id, _ptr(out)))
        return dict(learned=int(out[0]), plain=int(out[1]), judge=int(out[2]), fallbacks=int(out[3]),
                    disabled=bool(out[4]), judge_error=float(out[5]),
                    judge_error_per_variable=[float(x) for x in out[6:10]])

    def cgks_run_stage(self, mesh_id: int, stage: int):
        self._check(self._L.cgks_run_stage(self.h, mesh_id, stage))

    def cgks_launch_count(self, mesh_id: int, mode: int) -> int:
        out = C.c_int()
        self._check(self._L.cgks_launch_count(self.h, mesh_id, mode, C.byref(out)))
        return out.value

    def cgks_synchronize(self):
        self._check(self._L.cgks_synchronize(self.h))

    # ---- convenience -------------------------------------------------------------
    def setup(self, mesh_id: int, mesh: dict, winf, W, grad=None, levels: int | None = None):
        """Upload mesh + hierarchy, set the free stream and the initial state."""
        if mesh.get("mixed"):
            self.cgks_upload_mesh_mixed(mesh_id, mesh)
        else:
            self.cgks_upload_mesh(mesh_id, mesh)
        parents = mesh.get("parents", [])
        if levels is not None:
            parents = parents[: levels - 1]
        self.cgks_upload_hierarchy(mesh_id, parents)
        self.cgks_set_freestream(mesh_id, winf)
        self.cgks_init_state(mesh_id, W, grad)
