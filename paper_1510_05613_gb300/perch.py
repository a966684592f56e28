"""Thin ctypes binding of libperch.so (include/perch.h), same names.

Argument marshalling only: every step of successor evaluation and search runs
in the CUDA library. If the library is missing or fails to load this module
raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libperch.so")

PERCH_OK, PERCH_E_ARG, PERCH_E_CUDA, PERCH_E_OOM, PERCH_E_STATE, PERCH_E_TIMEOUT, PERCH_E_RANGE = 0, -1, -2, -3, -4, -5, -6
PERCH_E_DEVICE = -7
FLAG_CULLED, FLAG_INVALID, FLAG_TIMEOUT, FLAG_BAD_INDEX = 1, 2, 1 << 30, 1 << 31

OBJ = np.dtype([("mesh", np.uint16), ("iyaw", np.uint16), ("ix", np.int16), ("iy", np.int16)])
COST = np.dtype([("djr", np.int32), ("djo", np.int32), ("resid", np.int32), ("viol", np.int32),
                 ("n_new", np.int32), ("flags", np.uint32), ("n_vol", np.int32)])
# perch_icp (48 bytes): the planar motion, |M|, the last matching's pairs, the
# fits made, and PERCH_ICP_* (or flags bit 30 / 31)
ICP = np.dtype([("c", np.float64), ("s", np.float64), ("tx", np.float64), ("ty", np.float64),
                ("n_model", np.int32), ("n_corr", np.int32), ("iters", np.int32), ("status", np.uint32)])
PERCH_ICP_CONVERGED, PERCH_ICP_CAP, PERCH_ICP_FEW, PERCH_ICP_DEGENERATE = 0, 1, 2, 3

# names exported by the library (include/perch.h)
EXPORTS = ("perch_create", "perch_destroy", "perch_last_error", "perch_load_meshes", "perch_set_pose_grid",
           "perch_set_observation", "perch_eval_successors", "perch_eval_successors_dev", "perch_render",
           "perch_search", "perch_last_timing", "perch_eval_successors_noalloc", "perch_autotune",
           "perch_eval_graph", "perch_set_threads", "perch_set_scene", "perch_eval_successors_multi",
           "perch_search_multi", "perch_cnn_create", "perch_cnn_destroy", "perch_cnn_last_error",
           "perch_cnn_param_count", "perch_cnn_set_params", "perch_cnn_get_params", "perch_cnn_crops",
           "perch_cnn_forward", "perch_cnn_train_step", "perch_cnn_gradients", "perch_set_heuristic_net",
           "perch_cnn_set_tensor_path", "perch_cnn_tensor_status",
           "perch_set_shortcut", "perch_shortcut_stats", "perch_search_stats", "perch_search_times",
           "perch_set_wait_limit", "perch_set_share_renders", "perch_set_render_cache", "perch_last_phase_times", "perch_set_volumes",
           "perch_launch_config", "perch_set_symmetry", "perch_set_inline_pixels", "perch_set_bin_depth",
           "perch_launch_bin_depths", "perch_set_cost_stages", "perch_launch_cost_stages", "perch_icp_refine",
           "perch_icp_refine_dev")


class perch_mesh(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("n_verts", ctypes.c_int32), ("tris", ctypes.c_void_p),
                ("n_tris", ctypes.c_int32), ("vol_r", ctypes.c_float), ("vol_zlo", ctypes.c_float),
                ("vol_zhi", ctypes.c_float)]


class perch_volume(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("p", ctypes.c_float * 4),
                ("zlo", ctypes.c_float), ("zhi", ctypes.c_float), ("normals", ctypes.c_void_p)]


class perch_obj(ctypes.Structure):
    _fields_ = [("mesh", ctypes.c_uint16), ("iyaw", ctypes.c_uint16), ("ix", ctypes.c_int16), ("iy", ctypes.c_int16)]


class perch_search_params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("mesh_multiset", ctypes.c_void_p), ("w", ctypes.c_float),
                ("batch_states", ctypes.c_int32), ("time_limit_s", ctypes.c_double),
                ("max_expansions", ctypes.c_int64), ("heuristics", ctypes.c_int32)]


class perch_result(ctypes.Structure):
    _fields_ = [("objs", perch_obj * 16), ("n_objs", ctypes.c_int32), ("cost", ctypes.c_int64),
                ("expansions", ctypes.c_int64), ("successors", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("proven_optimal", ctypes.c_int32), ("found_seconds", ctypes.c_double),
                ("found_expansions", ctypes.c_int64)]


class PerchError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"perch error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libperch.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not built: run paper_1510_05613_gb300/build.py (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    P, I32, I64, F = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    sig = {
        "perch_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, P], ctypes.c_int),
        "perch_destroy": ([P], ctypes.c_int),
        "perch_last_error": ([P], ctypes.c_char_p),
        "perch_load_meshes": ([P, P, I32], ctypes.c_int),
        "perch_set_pose_grid": ([P, P, I32, P, I32, P, I32], ctypes.c_int),
        "perch_set_observation": ([P, P, I32, I32, P, P, F], ctypes.c_int),
        "perch_eval_successors": ([P, P, I32, P, I32, P, P, I64, I32, P], ctypes.c_int),
        "perch_eval_successors_dev": ([P, P, I32, P, I32, P, P, I64, I32, P], ctypes.c_int),
        "perch_render": ([P, P, I32, P, P], ctypes.c_int),
        "perch_search": ([P, P, P], ctypes.c_int),
        "perch_last_timing": ([P, P, P], ctypes.c_int),
        "perch_eval_successors_noalloc": ([P, P, I32, P, I32, P, P, I64, I32, P], ctypes.c_int),
        "perch_autotune": ([P, I32, P], ctypes.c_int),
        "perch_set_threads": ([P, I32, I32], ctypes.c_int),
        "perch_set_scene": ([P, I32, P], ctypes.c_int),
        "perch_eval_successors_multi": ([P, P, I32, P, P, P, I32, P, P, I64, P], ctypes.c_int),
        "perch_search_multi": ([P, I32, P, P, I64, P], ctypes.c_int),
        "perch_eval_graph": ([P, P, I32, P, I32, P, P, I64, I32, P, P], ctypes.c_int),
        "perch_cnn_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, P, I32, I32], ctypes.c_int),
        "perch_cnn_destroy": ([P], ctypes.c_int),
        "perch_cnn_last_error": ([P], ctypes.c_char_p),
        "perch_cnn_param_count": ([P, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "perch_cnn_set_params": ([P, P, I64], ctypes.c_int),
        "perch_cnn_get_params": ([P, P, I64], ctypes.c_int),
        "perch_cnn_crops": ([P, P, I32, P, P, I32, P, P, I64, P, P], ctypes.c_int),
        "perch_cnn_forward": ([P, P, P, I64, P], ctypes.c_int),
        "perch_cnn_set_tensor_path": ([P, I32], ctypes.c_int),
        "perch_cnn_tensor_status": ([P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "perch_cnn_train_step": ([P, P, P, P, I32, F, P], ctypes.c_int),
        "perch_cnn_gradients": ([P, P, P, P, I32, P, P, P], ctypes.c_int),
        "perch_set_heuristic_net": ([P, P, I32], ctypes.c_int),
        "perch_set_shortcut": ([P, I32], ctypes.c_int),
        "perch_set_wait_limit": ([P, I32], ctypes.c_int),
        "perch_set_volumes": ([P, P, I32], ctypes.c_int),
        "perch_launch_config": ([P, P, P, P], ctypes.c_int),
        "perch_set_inline_pixels": ([P, I32, I32], ctypes.c_int),
        "perch_set_bin_depth": ([P, I32, I32], ctypes.c_int),
        "perch_launch_bin_depths": ([P, P], ctypes.c_int),
        "perch_set_cost_stages": ([P, I32, I32], ctypes.c_int),
        "perch_launch_cost_stages": ([P, P], ctypes.c_int),
        "perch_icp_refine": ([P, P, I32, P, I32, P, P, I64, F, I32, P], ctypes.c_int),
        "perch_icp_refine_dev": ([P, P, I32, P, I32, P, P, I64, F, I32, P], ctypes.c_int),
        "perch_set_symmetry": ([P, P, I32], ctypes.c_int),
        "perch_set_share_renders": ([P, I32], ctypes.c_int),
        "perch_set_render_cache": ([P, I32], ctypes.c_int),
        "perch_last_phase_times": ([P, P, P], ctypes.c_int),
        "perch_search_stats": ([P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "perch_search_times": ([P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "perch_shortcut_stats": ([P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes, fn.restype = args, res
    _lib = lib
    return lib


def _ptr(a):
    return a.ctypes.data if a is not None and a.size else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Perch:
    """One library context (device memory, stream) on one GPU."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        h = ctypes.c_void_p()
        rc = self.lib.perch_create(ctypes.byref(h), device, stream)
        if rc != PERCH_OK:
            raise PerchError(rc, "perch_create failed")
        self.h = h
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            self.lib.perch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, ok=(PERCH_OK,)):
        if rc not in ok:
            raise PerchError(rc, self.lib.perch_last_error(self.h).decode())
        return rc

    # -- setup ---------------------------------------------------------
    def perch_load_meshes(self, meshes):
        arr = (perch_mesh * len(meshes))()
        keep = []
        for i, m in enumerate(meshes):
            v, t = _c(m.verts, np.float32), _c(m.tris, np.int32)
            keep += [v, t]
            arr[i] = perch_mesh(v.ctypes.data, m.n_verts, t.ctypes.data, m.n_tris, m.vol_r, m.vol_zlo, m.vol_zhi)
        return self._check(self.lib.perch_load_meshes(self.h, ctypes.addressof(arr), len(meshes)))

    def perch_set_pose_grid(self, grid):
        self.grid = grid  # for refined_pose
        xs, ys, cs = _c(grid.xs, np.float32), _c(grid.ys, np.float32), _c(grid.cos_sin, np.float32)
        return self._check(self.lib.perch_set_pose_grid(self.h, xs.ctypes.data, len(xs), ys.ctypes.data, len(ys),
                                                        cs.ctypes.data, cs.shape[0]))

    def perch_set_observation(self, depth, fxfycxcy, T_world_cam, delta: float):
        d = _c(depth, np.float32)
        H, W = d.shape
        k = _c(fxfycxcy, np.float32)
        T = _c(T_world_cam, np.float32).reshape(-1)
        return self._check(self.lib.perch_set_observation(self.h, d.ctypes.data, W, H, k.ctypes.data, T.ctypes.data,
                                                          delta))

    def setup(self, workload, exact_volumes: bool = False):
        """Meshes, pose grid and observation of a synth.Workload; with
        exact_volumes, V(O) is each mesh's closed form where it has one."""
        self.n_mesh = len(workload.meshes)
        self.perch_load_meshes(workload.meshes)
        if exact_volumes:
            self.perch_set_volumes(workload.meshes)
        self.perch_set_pose_grid(workload.grid)
        self.perch_set_observation(workload.depth, workload.cam.fxfycxcy, workload.cam.T_wc, workload.delta)
        self.H, self.W = workload.depth.shape

    # -- evaluation ----------------------------------------------------
    @staticmethod
    def pack_parents(parents):
        stride = max([1] + [len(p) for p in parents])
        P = np.zeros((max(1, len(parents)), stride), OBJ)
        plen = np.zeros(max(1, len(parents)), np.int32)
        for i, p in enumerate(parents):
            p = np.asarray(p, OBJ)
            P[i, :len(p)] = p
            plen[i] = len(p)
        return P, plen, stride

    def perch_eval_successors(self, parents, hyp_parent, hyps, K_total: int):
        """Host arrays in, structured COST array out. ``parents``: list of
        object arrays (partial assignments)."""
        P, plen, stride = self.pack_parents(parents)
        hp = _c(hyp_parent, np.int32)
        h = _c(hyps, OBJ)
        out = np.zeros(len(h), COST)
        self._check(self.lib.perch_eval_successors(self.h, P.ctypes.data, stride, plen.ctypes.data, len(plen),
                                                   _ptr(hp), _ptr(h), len(h), K_total, _ptr(out)))
        return out

    def perch_eval_successors_dev(self, parents_t, stride: int, plen_t, hyp_parent_t, hyps_t, K_total: int, out_t):
        """Device buffers (torch tensors) in and out; enqueued on the context's stream."""
        return self._check(self.lib.perch_eval_successors_dev(
            self.h, parents_t.data_ptr(), stride, plen_t.data_ptr(), plen_t.numel(), hyp_parent_t.data_ptr(),
            hyps_t.data_ptr(), hyp_parent_t.numel(), K_total, out_t.data_ptr()))

    def perch_eval_successors_noalloc(self, parents_t, stride: int, plen_t, hyp_parent_t, hyps_t, K_total: int,
                                      out_t):
        """As perch_eval_successors_dev, with the library's fixed scratch array
        instead of context-allocated scratch (the call allocates nothing)."""
        return self._check(self.lib.perch_eval_successors_noalloc(
            self.h, parents_t.data_ptr(), stride, plen_t.data_ptr(), plen_t.numel(), hyp_parent_t.data_ptr(),
            hyps_t.data_ptr(), hyp_parent_t.numel(), K_total, out_t.data_ptr()))

    def perch_icp_refine(self, parents, hyp_parent, hyps, radius: float = 0.02, max_iter: int = 20):
        """ICP refinement of each hypothesis's new object against its parent
        (host arrays in, structured ICP array out)."""
        P, plen, stride = self.pack_parents(parents)
        hp = _c(hyp_parent, np.int32)
        h = _c(hyps, OBJ)
        out = np.zeros(len(h), ICP)
        self._check(self.lib.perch_icp_refine(self.h, P.ctypes.data, stride, plen.ctypes.data, len(plen), _ptr(hp),
                                              _ptr(h), len(h), radius, max_iter, _ptr(out)))
        return out

    def perch_icp_refine_dev(self, parents_t, stride: int, plen_t, hyp_parent_t, hyps_t, radius: float,
                             max_iter: int, out_t):
        """Device buffers (torch tensors; out_t holds 48 bytes per hypothesis)
        in and out; enqueued on the context's stream."""
        return self._check(self.lib.perch_icp_refine_dev(
            self.h, parents_t.data_ptr(), stride, plen_t.data_ptr(), plen_t.numel(), hyp_parent_t.data_ptr(),
            hyps_t.data_ptr(), hyp_parent_t.numel(), radius, max_iter, out_t.data_ptr()))

    def perch_refine_scene(self, objs, radius: float = 0.02, max_iter: int = 20):
        """ICP of each object of a scene against all the others: its model
        set is then its visible part in the whole scene, which for a scene of
        the MSGT is its non-occluded part when it was added (the objects
        added after it lie behind it or beside it, Eq. (3)), in any order of
        objs. Returns (records, [(mesh, x, y, yaw)])."""
        objs = np.asarray(objs, OBJ)
        others = [np.concatenate([objs[:k], objs[k + 1:]]) for k in range(len(objs))]
        recs = self.perch_icp_refine(others, np.arange(len(objs)), objs, radius, max_iter)
        return recs, [refined_pose(self.grid, o, r) for o, r in zip(objs, recs)]

    def perch_autotune(self, n_sample: int = 2048):
        """Pick the CTA width per mesh by timing; returns the choices."""
        out = (ctypes.c_int32 * 65536)()
        self._check(self.lib.perch_autotune(self.h, n_sample, out))
        return [int(out[i]) for i in range(self.n_mesh)]

    def perch_set_threads(self, threads: int, mesh: int = -1):
        return self._check(self.lib.perch_set_threads(self.h, mesh, threads))

    def perch_eval_graph(self, parents_t, stride: int, plen_t, hyp_parent_t, hyps_t, K_total: int, out_t,
                         out_host=None):
        """As perch_eval_successors_dev, captured once into a CUDA graph and
        replayed; out_host: optional pinned host array (torch, uint8/int32)."""
        return self._check(self.lib.perch_eval_graph(
            self.h, parents_t.data_ptr(), stride, plen_t.data_ptr(), plen_t.numel(), hyp_parent_t.data_ptr(),
            hyps_t.data_ptr(), hyp_parent_t.numel(), K_total, out_t.data_ptr(),
            None if out_host is None else out_host.data_ptr()))

    def perch_set_scene(self, scene: int, depth):
        d = _c(depth, np.float32)
        return self._check(self.lib.perch_set_scene(self.h, scene, d.ctypes.data))

    def perch_eval_successors_multi(self, parents, parent_scene, parent_K, hyp_parent, hyps):
        P, plen, stride = self.pack_parents(parents)
        ps, pk = _c(parent_scene, np.int32), _c(parent_K, np.int32)
        hp, h = _c(hyp_parent, np.int32), _c(hyps, OBJ)
        out = np.zeros(len(h), COST)
        self._check(self.lib.perch_eval_successors_multi(self.h, P.ctypes.data, stride, plen.ctypes.data,
                                                         ps.ctypes.data, pk.ctypes.data, len(plen), _ptr(hp),
                                                         _ptr(h), len(h), _ptr(out)))
        return out

    def perch_search_multi(self, scenes, multisets, batch_states: int = 1, max_hyps_per_launch: int = 1 << 22,
                           time_limit_s: float = 0.0, w: float = 1.0, heuristics: int = 0):
        n = len(scenes)
        keep = [_c(ms, np.uint16) for ms in multisets]
        params = (perch_search_params * n)()
        for i, ms in enumerate(keep):
            params[i] = perch_search_params(len(ms), ms.ctypes.data, w, batch_states, time_limit_s, 0, heuristics)
        sc = _c(scenes, np.int32)
        res = (perch_result * n)()
        rc = self.lib.perch_search_multi(self.h, n, sc.ctypes.data, params, max_hyps_per_launch, res)
        self._check(rc, ok=(PERCH_OK, PERCH_E_TIMEOUT))
        return [self._result(res[i], PERCH_OK) for i in range(n)]

    @staticmethod
    def _result(r, rc):
        objs = np.array([(r.objs[i].mesh, r.objs[i].iyaw, r.objs[i].ix, r.objs[i].iy) for i in range(r.n_objs)], OBJ)
        key = tuple(sorted((int(o["mesh"]), int(o["ix"]), int(o["iy"]), int(o["iyaw"])) for o in objs))
        return {"cost": int(r.cost), "key": key, "objs": objs, "expansions": int(r.expansions),
                "successors": int(r.successors), "seconds": float(r.seconds),
                "proven_optimal": bool(r.proven_optimal), "status": rc,
                "found_seconds": float(r.found_seconds), "found_expansions": int(r.found_expansions)}

    def perch_cnn_crops(self, parents, hyp_parent, hyps, parent_scene=None):
        """Network inputs of the hypotheses: (crops, onehot) as torch device
        tensors, (n, 64, 64, 2) bfloat16 and (n,) int32."""
        import torch
        P, plen, stride = self.pack_parents(parents)
        hp, h = _c(hyp_parent, np.int32), _c(hyps, OBJ)
        ps = None if parent_scene is None else _c(parent_scene, np.int32)
        crops = torch.empty((len(h), 64, 64, 2), dtype=torch.bfloat16, device="cuda")
        onehot = torch.empty(len(h), dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        self._check(self.lib.perch_cnn_crops(self.h, P.ctypes.data, stride, plen.ctypes.data, _ptr(ps), len(plen),
                                             _ptr(hp), _ptr(h), len(h), crops.data_ptr() if len(h) else None,
                                             onehot.data_ptr() if len(h) else None))
        return crops, onehot

    def perch_set_heuristic_net(self, net, n_candidates: int = 16):
        """Attach a PerchCNN (None detaches) for search heuristic bit 2."""
        self._net = net  # keep it alive while attached
        return self._check(self.lib.perch_set_heuristic_net(self.h, None if net is None else net.h, n_candidates))

    def perch_set_share_renders(self, on: bool):
        """One render per distinct pose of a batch (on by default)."""
        return self._check(self.lib.perch_set_share_renders(self.h, 1 if on else 0))

    def perch_set_render_cache(self, on: bool):
        """Keep each pose's render across evaluations until the observation,
        the scenes or the pose tables change (records unchanged)."""
        return self._check(self.lib.perch_set_render_cache(self.h, 1 if on else 0))

    def perch_last_phase_times(self):
        """(ms per phase [prep, grouping, render, cost], shared renders used)."""
        ms = np.zeros(4, np.float32)
        shared = ctypes.c_int32(0)
        self._check(self.lib.perch_last_phase_times(self.h, ms.ctypes.data, ctypes.byref(shared)))
        return ms.astype(np.float64), bool(shared.value)

    def perch_set_symmetry(self, meshes):
        """The search places each mesh only at yaws that are distinct modulo
        its rotational symmetry (synth.Mesh.sym); None: every yaw."""
        if meshes is None:
            return self._check(self.lib.perch_set_symmetry(self.h, None, 0))
        sym = np.array([int(getattr(m, "sym", 1)) for m in meshes], np.int32)
        return self._check(self.lib.perch_set_symmetry(self.h, sym.ctypes.data, len(sym)))

    def perch_launch_config(self):
        """(render CTA width, render inline limit, cost CTA width) per mesh, now in use."""
        r = np.zeros(self.n_mesh, np.int32)
        i = np.zeros(self.n_mesh, np.int32)
        c = np.zeros(self.n_mesh, np.int32)
        self._check(self.lib.perch_launch_config(self.h, r.ctypes.data, i.ctypes.data, c.ctypes.data))
        return r.tolist(), i.tolist(), c.tolist()

    def perch_set_inline_pixels(self, inline_pixels: int, mesh: int = -1):
        """The render's inline limit (8, 16 or 32) for one mesh or all."""
        return self._check(self.lib.perch_set_inline_pixels(self.h, mesh, int(inline_pixels)))

    def perch_set_bin_depth(self, depth: int, mesh: int = -1):
        """Depth (32, 64 or 128) of the render's bin of larger triangles, for one mesh or all."""
        return self._check(self.lib.perch_set_bin_depth(self.h, mesh, int(depth)))

    def perch_launch_bin_depths(self):
        """The bin depth in use per mesh."""
        out = np.zeros(self.n_mesh, np.int32)
        self._check(self.lib.perch_launch_bin_depths(self.h, out.ctypes.data))
        return out.tolist()

    def perch_set_cost_stages(self, stages: int, mesh: int = -1):
        """Stage buffers (1 or 2) of the cost launch, for one mesh or all."""
        return self._check(self.lib.perch_set_cost_stages(self.h, mesh, int(stages)))

    def perch_launch_cost_stages(self):
        """The cost launch's stage buffers in use per mesh."""
        out = np.zeros(self.n_mesh, np.int32)
        self._check(self.lib.perch_launch_cost_stages(self.h, out.ctypes.data))
        return out.tolist()

    def perch_set_volumes(self, meshes):
        """V(O) per mesh from each synth.Mesh's closed-form `volume` (None:
        the inscribed cylinder); meshes = None restores the cylinders."""
        if meshes is None:
            return self._check(self.lib.perch_set_volumes(self.h, None, 0))
        arr = (perch_volume * len(meshes))()
        keep = []
        for i, m in enumerate(meshes):
            v = getattr(m, "volume", None)
            if v is None:
                continue
            nr = _c(v.normals, np.float32)
            keep.append(nr)
            arr[i].kind, arr[i].n = int(v.kind), int(v.n)
            for k in range(4):
                arr[i].p[k] = float(np.float32(v.p[k]))
            arr[i].zlo, arr[i].zhi = float(v.zlo), float(v.zhi)
            arr[i].normals = nr.ctypes.data if nr.size else None
        return self._check(self.lib.perch_set_volumes(self.h, arr, len(meshes)))

    def perch_set_wait_limit(self, polls: int):
        """Poll bound of the evaluation kernel's first wait per bulk copy
        (< 0: the default); 0 makes every such wait give up at once."""
        return self._check(self.lib.perch_set_wait_limit(self.h, int(polls)))

    def perch_set_shortcut(self, on: bool):
        """Exact shortcut for hypotheses far from the observation and the parent (on by default)."""
        return self._check(self.lib.perch_set_shortcut(self.h, 1 if on else 0))

    def perch_shortcut_stats(self):
        """(hypotheses that took the shortcut, hypotheses) of the last evaluation."""
        a, b = ctypes.c_int64(0), ctypes.c_int64(0)
        self._check(self.lib.perch_shortcut_stats(self.h, ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    def perch_search_stats(self):
        """Learned queue cost of the last search: (seconds, states scored, crops)."""
        a, b, c = ctypes.c_double(0), ctypes.c_int64(0), ctypes.c_int64(0)
        self._check(self.lib.perch_search_stats(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return float(a.value), int(b.value), int(c.value)

    def perch_search_times(self):
        """Wall seconds of the last search: (device evaluation, absorbing records, selecting states)."""
        a, b, c = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
        self._check(self.lib.perch_search_times(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return float(a.value), float(b.value), float(c.value)

    def perch_render(self, objs):
        o = _c(objs, OBJ)
        out = np.empty((self.H, self.W), np.float32)
        n = ctypes.c_int64(0)
        self._check(self.lib.perch_render(self.h, _ptr(o), len(o), out.ctypes.data, ctypes.byref(n)))
        return out, int(n.value)

    def perch_last_timing(self):
        """(prep_ms, eval_ms) of the last evaluation, from CUDA events."""
        a, b = ctypes.c_float(0), ctypes.c_float(0)
        self._check(self.lib.perch_last_timing(self.h, ctypes.byref(a), ctypes.byref(b)))
        return float(a.value), float(b.value)

    def perch_search(self, mesh_multiset, w: float = 1.0, batch_states: int = 8, time_limit_s: float = 0.0,
                     max_expansions: int = 0, heuristics: int = 0):
        ms = _c(mesh_multiset, np.uint16)
        p = perch_search_params(len(ms), ms.ctypes.data, w, batch_states, time_limit_s, max_expansions, heuristics)
        r = perch_result()
        rc = self.lib.perch_search(self.h, ctypes.byref(p), ctypes.byref(r))
        self._check(rc, ok=(PERCH_OK, PERCH_E_TIMEOUT))
        objs = np.array([(r.objs[i].mesh, r.objs[i].iyaw, r.objs[i].ix, r.objs[i].iy) for i in range(r.n_objs)], OBJ)
        key = tuple(sorted((int(o["mesh"]), int(o["ix"]), int(o["iy"]), int(o["iyaw"])) for o in objs))
        return {"cost": int(r.cost), "key": key, "objs": objs, "expansions": int(r.expansions),
                "successors": int(r.successors), "seconds": float(r.seconds),
                "proven_optimal": bool(r.proven_optimal), "status": rc,
                "found_seconds": float(r.found_seconds), "found_expansions": int(r.found_expansions)}


class PerchCNN:
    """The learned heuristic's network on one GPU (perch_cnn_* entry points).
    Device arrays are torch tensors; calls are ordered with torch's work by
    synchronising the device around them."""

    def __init__(self, n_onehot: int, max_batch: int = 256, device: int = 0, stream=None):
        """``stream``: a torch.cuda.Stream (or raw handle) to run on; None: the
        network's own stream."""
        self.lib = load()
        h = ctypes.c_void_p()
        handle = getattr(stream, "cuda_stream", stream)
        rc = self.lib.perch_cnn_create(ctypes.byref(h), device, handle or None, n_onehot, max_batch)
        if rc != PERCH_OK:
            raise PerchError(rc, "perch_cnn_create failed")
        self.h = h
        self.n_onehot = n_onehot
        self.max_batch = max_batch
        n = ctypes.c_int64(0)
        self._check(self.lib.perch_cnn_param_count(self.h, ctypes.byref(n)))
        self.n_params = int(n.value)

    def close(self):
        if getattr(self, "h", None):
            self.lib.perch_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != PERCH_OK:
            raise PerchError(rc, self.lib.perch_cnn_last_error(self.h).decode())
        return rc

    def perch_cnn_set_params(self, params):
        p = _c(np.concatenate([np.asarray(a, np.float32).reshape(-1) for a in params]), np.float32)
        return self._check(self.lib.perch_cnn_set_params(self.h, p.ctypes.data, p.size))

    def perch_cnn_get_params(self) -> np.ndarray:
        p = np.empty(self.n_params, np.float32)
        self._check(self.lib.perch_cnn_get_params(self.h, p.ctypes.data, p.size))
        return p

    def perch_cnn_set_tensor_path(self, path: int):
        """0: mma.sync convolutions (default); 1: tcgen05 for the forward 3x3 convolutions 2-4."""
        self._check(self.lib.perch_cnn_set_tensor_path(self.h, int(path)))

    def perch_cnn_tensor_status(self):
        """(tensor path, 1 if a bounded wait of the tcgen05 kernel gave up)."""
        a, b = ctypes.c_int32(0), ctypes.c_int32(0)
        self._check(self.lib.perch_cnn_tensor_status(self.h, ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    def perch_cnn_forward(self, crops, onehot):
        import torch
        pred = torch.empty(crops.shape[0], dtype=torch.float32, device=crops.device)
        torch.cuda.synchronize()
        self._check(self.lib.perch_cnn_forward(self.h, crops.data_ptr(), onehot.data_ptr(), crops.shape[0],
                                               pred.data_ptr()))
        torch.cuda.synchronize()
        return pred

    def perch_cnn_train_step(self, crops, onehot, target, lr: float, loss=None):
        """Enqueue one Adam step; ``loss`` (a device float32 tensor of one
        element, optional) receives the batch loss."""
        return self._check(self.lib.perch_cnn_train_step(self.h, crops.data_ptr(), onehot.data_ptr(),
                                                         target.data_ptr(), crops.shape[0], lr,
                                                         None if loss is None else loss.data_ptr()))

    def perch_cnn_gradients(self, crops, onehot, target):
        """(packed gradients, loss, predictions) on the host."""
        import torch
        n = crops.shape[0]
        g = np.empty(self.n_params, np.float32)
        loss = ctypes.c_float(0)
        pred = np.empty(n, np.float32)
        torch.cuda.synchronize()
        self._check(self.lib.perch_cnn_gradients(self.h, crops.data_ptr(), onehot.data_ptr(), target.data_ptr(), n,
                                                 g.ctypes.data, ctypes.byref(loss), pred.ctypes.data))
        return g, float(loss.value), pred

    def synchronize(self):
        import torch
        torch.cuda.synchronize()


def refined_pose(grid, obj, rec):
    """(mesh, x, y, yaw) of a grid object moved by an ICP record's motion:
    (x, y) turned and shifted, the yaw turned by atan2(s, c)."""
    import math
    x, y = float(grid.xs[int(obj["ix"])]), float(grid.ys[int(obj["iy"])])
    c0, s0 = (float(v) for v in grid.cos_sin[int(obj["iyaw"])])
    c, s = float(rec["c"]), float(rec["s"])
    return (int(obj["mesh"]), c * x - s * y + float(rec["tx"]), s * x + c * y + float(rec["ty"]),
            math.atan2(s0, c0) + math.atan2(s, c))


def records(out) -> np.ndarray:
    """COST structured array -> (n, 7) int64 (djr, djo, resid, viol, n_new, flags, n_vol)."""
    return np.stack([out[f].astype(np.int64) for f in COST.names], 1)
