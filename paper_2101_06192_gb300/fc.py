"""Thin ctypes binding of libfc.so (include/fc.h).  Argument marshalling only:
every step of the computation runs in the library's CUDA kernels.  PyTorch is
used for device memory and the current CUDA stream.

Raises FcError on any non-OK status.  There is no CPU path: if the library
cannot be built or loaded, importing the handle fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

_lib = None

FC_OK, FC_EINVAL, FC_ENOMEM, FC_ECUDA, FC_ENOCONV, FC_ETIMEOUT, FC_EOVERFLOW = range(7)
FC_HOST_PTRS, FC_DEVICE_PTRS = 0, 1


class FcError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


def lib():
    """Load (building first if stale) the in-tree libfc.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P, I32, I64, U32, U64, D = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_double)
        sig = {
            "fc_build_augmented": ([I32, I64, P, P, P, P, I32, U32, P, ctypes.POINTER(P)], ctypes.c_int),
            "fc_graph_info": ([P, P, P, P, P], ctypes.c_int),
            "fc_build_batch": ([I32, P, I64, P, P, P, P, U32, P, ctypes.POINTER(P)], ctypes.c_int),
            "fc_batch_latency": ([P, P], ctypes.c_int),
            "fc_set_sampler_shape": ([P, I32, I32, I32, I32], ctypes.c_int),
            "fc_sampler_last_shape": ([P, P, P, P], ctypes.c_int),
            "fc_set_start_order": ([P, I32], ctypes.c_int),
            "fc_set_sampler_kernel": ([P, I32], ctypes.c_int),
            "fc_sampler_last_kernel": ([P], I32),
            "fc_set_sampler_pops": ([P, I32], ctypes.c_int),
            "fc_set_sampler_bitmap": ([P, I32], ctypes.c_int),
            "fc_set_sampler_cluster": ([P, I32], ctypes.c_int),
            "fc_sampler_last_cluster": ([P], I32),
            "fc_sampler_counters": ([P, P, I32], ctypes.c_int),
            "fc_sample_usts": ([P, U64, I64, I64, P, P, P, U64, P, P], ctypes.c_int),
            "fc_sampler_stats": ([P, P, P], ctypes.c_int),
            "fc_sample_usts_async": ([P, U64, I64, I64, P, P, P, U64, P, P], ctypes.c_int),
            "fc_sampler_check": ([P, P], ctypes.c_int),
            "fc_stack_entries": ([P, I32, U64, U32, I64, P, P, P, P], ctypes.c_int),
            "fc_solve": ([P, I32, P, P, I32, D, I32, P, P], ctypes.c_int),
            "fc_pivot_solve": ([P, I32, P, D, I32, P, P], ctypes.c_int),
            "fc_forest_farness": ([P, I32, P, P, P, P, I64, P, P, P, P], ctypes.c_int),
            "fc_forest_farness_noalloc": ([P, I32, P, P, P, P, I64, P, P, P, P], ctypes.c_int),
            "fc_p_root": ([P, I32, P, P], ctypes.c_int),
            "fc_top_k": ([P, I32, I32, P, P], ctypes.c_int),
            "fc_tree_roots": ([P, I32, I64, P, P, P], ctypes.c_int),
            "fc_rb_accumulate": ([P, I32, P, I64, P, P], ctypes.c_int),
            "fc_rb_diag": ([P, I32, I64, P, P], ctypes.c_int),
            "fc_farness_from_diag": ([P, P, P, P, P], ctypes.c_int),
            "fc_group_closeness": ([P, I32, I32, D, P, P, P], ctypes.c_int),
            "fc_root_counts": ([P, I32, I64, P, I32, P, P], ctypes.c_int),
            "fc_mlp_param_count": ([], I32),
            "fc_vertex_features": ([P, I32, P, P], ctypes.c_int),
            "fc_mlp_forward": ([P, I32, P, P, P, P], ctypes.c_int),
            "fc_mlp_loss_grad": ([P, I32, P, P, P, P, P, P], ctypes.c_int),
            "fc_mlp_loss_grad_acc": ([P, I32, P, P, P, ctypes.c_float, I32, P, P, P], ctypes.c_int),
            "fc_mlp_adam": ([P, P, P, P, I32, I32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, P], ctypes.c_int),
            "fc_tau_for": ([D, D, D, I64], I64),
            "fc_build_rooted": ([I32, I64, P, P, P, I32, U32, P, ctypes.POINTER(P)], ctypes.c_int),
            "fc_bfs_tree": ([P, P, P, P], ctypes.c_int),
            "fc_resistance_accumulate": ([P, P, I64, P, P], ctypes.c_int),
            "fc_laplacian_solve": ([P, P, P, I32, D, I32, P, P], ctypes.c_int),
            "fc_electrical_closeness": ([P, P, P, I64, P, P, P, P, P, P], ctypes.c_int),
            "fc_sample_usts_ex": ([P, U64, I64, I64, P, P, P, P, U64, P, P], ctypes.c_int),
            "fc_sample_usts_forest": ([P, U64, I64, I64, P, P, P, P, P, P, U64, P, P], ctypes.c_int),
            "fc_visit_diag": ([P, I32, P, I64, P, P], ctypes.c_int),
            "fc_destroy": ([P], None),
            "fc_status_str": ([ctypes.c_int], ctypes.c_char_p),
            "fc_last_error_message": ([], ctypes.c_char_p),
            "fc_launch_count": ([], ctypes.c_uint64),
            "fc_release_scratch": ([], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != FC_OK:
        L = lib()
        detail = L.fc_last_error_message().decode() or L.fc_status_str(status).decode()
        raise FcError(status, where, detail)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_tensor(t, dtype, n, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
            and t.numel() >= n):
        raise ValueError(f"{name}: expected a contiguous CUDA {dtype} tensor with >= {n} elements")
    return t


class Graph:
    """G* over one CSR graph for one or more alphas (fc_build_augmented)."""

    def __init__(self, rowptr, colidx, w=None, alphas=(1.0,), stream=None):
        L = lib()
        alphas = np.ascontiguousarray(np.atleast_1d(np.asarray(alphas, dtype=np.float64)))
        on_dev = isinstance(rowptr, torch.Tensor) and rowptr.is_cuda
        if on_dev:
            rp = rowptr.to(torch.int64).contiguous()
            ci = colidx.to(torch.int32).contiguous()
            ww = None if w is None else w.to(torch.float32).contiguous()
            flags = FC_DEVICE_PTRS
        else:
            rp = np.ascontiguousarray(rowptr, dtype=np.int64)
            ci = np.ascontiguousarray(colidx, dtype=np.int32)
            ww = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
            flags = FC_HOST_PTRS
        n = int(rp.shape[0]) - 1
        nnz = int(ci.shape[0])
        h = ctypes.c_void_p()
        _check(L.fc_build_augmented(n, nnz, _ptr(rp), _ptr(ci), _ptr(ww), _ptr(alphas), int(alphas.size),
                                    flags, _stream(stream), ctypes.byref(h)), "fc_build_augmented")
        self._h = h
        self.n = n
        self.nnz = nnz
        self.alphas = alphas.copy()
        self.n_alpha = int(alphas.size)
        self.weighted = w is not None

    @classmethod
    def batch(cls, union_csr, vertex_offsets, graph_alphas, stream=None):
        """fc_build_batch: graphs as one block-diagonal CSR (host arrays), one alpha each."""
        self = cls.__new__(cls)
        voff = np.ascontiguousarray(vertex_offsets, dtype=np.int64)
        ga = np.ascontiguousarray(graph_alphas, dtype=np.float64)
        rp = np.ascontiguousarray(union_csr.rowptr, dtype=np.int64)
        ci = np.ascontiguousarray(union_csr.colidx, dtype=np.int32)
        ww = None if union_csr.w is None else np.ascontiguousarray(union_csr.w, dtype=np.float32)
        h = ctypes.c_void_p()
        _check(lib().fc_build_batch(int(ga.size), _ptr(voff), int(ci.shape[0]), _ptr(rp), _ptr(ci), _ptr(ww), _ptr(ga),
                                    FC_HOST_PTRS, _stream(stream), ctypes.byref(h)), "fc_build_batch")
        self._h = h
        self.n = int(rp.shape[0]) - 1
        self.nnz = int(ci.shape[0])
        self.alphas = np.ones(1)
        self.n_alpha = 1
        self.weighted = ww is not None
        self.num_graphs = int(ga.size)
        self.vertex_offsets = voff.copy()
        return self

    @classmethod
    def rooted(cls, g, root: int, stream=None):
        """fc_build_rooted: G (host CSR) with walks whose only exit is ``root``
        (uniform spanning trees of G rooted there) and root's BFS tree."""
        self = cls.__new__(cls)
        rp = np.ascontiguousarray(g.rowptr, dtype=np.int64)
        ci = np.ascontiguousarray(g.colidx, dtype=np.int32)
        ww = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.float32)
        h = ctypes.c_void_p()
        _check(lib().fc_build_rooted(int(rp.shape[0]) - 1, int(ci.shape[0]), _ptr(rp), _ptr(ci), _ptr(ww), int(root),
                                     FC_HOST_PTRS, _stream(stream), ctypes.byref(h)), "fc_build_rooted")
        self._h = h
        self.n = int(rp.shape[0]) - 1
        self.nnz = int(ci.shape[0])
        self.alphas = np.ones(1)
        self.n_alpha = 1
        self.weighted = ww is not None
        self.root = int(root)
        return self

    def bfs_tree(self, stream=None):
        """fc_bfs_tree: (parent, depth) of the root's breadth-first tree."""
        dev = torch.device("cuda", torch.cuda.current_device())
        par = torch.empty(self.n, dtype=torch.int32, device=dev)
        dep = torch.empty(self.n, dtype=torch.int32, device=dev)
        _check(lib().fc_bfs_tree(self._h, _ptr(par), _ptr(dep), _stream(stream)), "fc_bfs_tree")
        return par, dep

    def resistance_accumulate(self, parents, acc=None, stream=None):
        """fc_resistance_accumulate over parents [T, n]; acc (int64 [n]) accumulates."""
        parents = parents.reshape(-1, self.n).to(torch.int32).contiguous()
        if acc is None:
            acc = torch.zeros(self.n, dtype=torch.int64, device=parents.device)
        _dev_tensor(acc, torch.int64, self.n, "acc")
        _check(lib().fc_resistance_accumulate(self._h, _ptr(parents), int(parents.shape[0]), _ptr(acc),
                                              _stream(stream)), "fc_resistance_accumulate")
        return acc

    def laplacian_solve(self, b, x=None, rel_tol: float = 1e-9, max_iter: int = 20000, stream=None):
        """fc_laplacian_solve: L^+ b for b of shape [n] or [m, n] (FP64, CUDA).  Returns (x, iters)."""
        b2 = b.reshape(-1, self.n).contiguous()
        x = torch.zeros_like(b2) if x is None else x.reshape(-1, self.n)
        it = ctypes.c_int32()
        _check(lib().fc_laplacian_solve(self._h, _ptr(b2), _ptr(x), int(b2.shape[0]), float(rel_tol), int(max_iter),
                                        ctypes.byref(it), _stream(stream)), "fc_laplacian_solve")
        return x.reshape(b.shape), it.value

    def electrical_closeness(self, acc, trees: int, x_pivot, visits=None, stream=None):
        """fc_electrical_closeness from path-sum totals ``acc`` or (acc None) visit
        totals ``visits``: (r^(root, .), diag(L^+), farness, closeness), FP64 [n] each."""
        dev = x_pivot.device
        outs = [torch.empty(self.n, dtype=torch.float64, device=dev) for _ in range(4)]
        _check(lib().fc_electrical_closeness(self._h, _ptr(acc), _ptr(visits), int(trees), _ptr(x_pivot.contiguous()),
                                             *[_ptr(o) for o in outs], _stream(stream)), "fc_electrical_closeness")
        return tuple(outs)

    def batch_latency_ms(self):
        out = np.zeros(self.num_graphs, dtype=np.float64)
        _check(lib().fc_batch_latency(self._h, _ptr(out)), "fc_batch_latency")
        return out

    @classmethod
    def from_csr(cls, g, alphas=(1.0,), stream=None):
        """From any object with rowptr/colidx/w numpy arrays (host copy path)."""
        return cls(g.rowptr, g.colidx, g.w, alphas, stream)

    def close(self):
        if getattr(self, "_h", None):
            lib().fc_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_shape(self, walkers_per_tree: int = 0, max_trees_resident: int = 0, smem: int = 0, regs: int = 0):
        _check(lib().fc_set_sampler_shape(self._h, walkers_per_tree, max_trees_resident, smem, regs),
               "fc_set_sampler_shape")

    START_ORDERS = {"degree": 0, "degree_desc": 1, "id": 2, "id_desc": 3, "auto": 4}

    def set_start_order(self, order):
        """fc_set_start_order: "auto" (default), "degree", "degree_desc", "id", "id_desc"
        (or the integer code; True/False select descending/ascending degree)."""
        if isinstance(order, bool):
            code = int(order)
        elif isinstance(order, str):
            code = self.START_ORDERS[order]
        else:
            code = int(order)
        _check(lib().fc_set_start_order(self._h, code), "fc_set_start_order")

    kernel_pref = 0

    def set_kernel(self, kernel: int = 0):
        """fc_set_sampler_kernel: 0 automatic, 1 CSR-walk, 2 edge-record."""
        _check(lib().fc_set_sampler_kernel(self._h, int(kernel)), "fc_set_sampler_kernel")
        self.kernel_pref = int(kernel)

    def set_pops(self, mode: int = 0):
        """fc_set_sampler_pops: 0 automatic, 1 walk every cycle, 2 pop short cycles from the ring."""
        _check(lib().fc_set_sampler_pops(self._h, int(mode)), "fc_set_sampler_pops")

    def set_bitmap(self, mode: int = 0):
        """fc_set_sampler_bitmap: 0 automatic, 1 state flags, 2 shared memory, 3 global memory."""
        _check(lib().fc_set_sampler_bitmap(self._h, int(mode)), "fc_set_sampler_bitmap")

    def set_cluster(self, ctas_per_tree: int = 0):
        """fc_set_sampler_cluster: CTAs per tree (0 automatic, 1, 2, 4 or 8)."""
        _check(lib().fc_set_sampler_cluster(self._h, int(ctas_per_tree)), "fc_set_sampler_cluster")

    def last_cluster(self) -> int:
        return int(lib().fc_sampler_last_cluster(self._h))

    def last_kernel(self) -> int:
        return int(lib().fc_sampler_last_kernel(self._h))

    COUNTERS = ("iterations", "claims", "tree_hits", "confirms", "conflict_waits", "release_waits",
                "releases", "pop_steps", "tops_k_gt_0", "idle_lane_iterations")

    def sampler_counters(self):
        out = (ctypes.c_uint64 * 10)()
        _check(lib().fc_sampler_counters(self._h, out, 10), "fc_sampler_counters")
        return dict(zip(self.COUNTERS, [int(v) for v in out]))

    def last_shape(self):
        w, r, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().fc_sampler_last_shape(self._h, ctypes.byref(w), ctypes.byref(r), ctypes.byref(c)),
               "fc_sampler_last_shape")
        return {"walkers_per_tree": w.value, "regs": r.value, "ctas": c.value}

    def sample_async(self, seed: int, tau: int, R, C=None, tree_offset: int = 0, stream=None):
        """fc_sample_usts_async (capturable; errors via check())."""
        _check(lib().fc_sample_usts_async(self._h, int(seed) & (2**64 - 1), int(tau), int(tree_offset), _ptr(R),
                                          _ptr(C), None, 0, None, _stream(stream)), "fc_sample_usts_async")

    def check(self, stream=None):
        _check(lib().fc_sampler_check(self._h, _stream(stream)), "fc_sampler_check")

    def sample(self, seed: int, tau: int, tree_offset: int = 0, R=None, C=None, with_C: bool = True,
               want_parents: bool = False, want_steps: bool = False, max_steps_per_tree: int = 0,
               visits=None, want_visits: bool = False, want_roots: bool = False, stream=None):
        """fc_sample_usts (fc_sample_usts_ex when visit totals are wanted,
        fc_sample_usts_forest when forest roots and depths are).  R, C and
        visits accumulate (allocated zeroed when not given)."""
        dev = torch.device("cuda", torch.cuda.current_device())
        na, n = self.n_alpha, self.n
        if R is None:
            R = torch.zeros(na * n, dtype=torch.int32, device=dev)
        _dev_tensor(R, torch.int32, na * n, "R")
        if C is None and with_C:
            C = torch.zeros(na * n, dtype=torch.int32, device=dev)
        if C is not None:
            _dev_tensor(C, torch.int32, na * n, "C")
        parents = torch.empty(na * tau * n, dtype=torch.int32, device=dev) if want_parents else None
        nrow = getattr(self, "num_graphs", 0) or na
        steps = torch.zeros(nrow * tau, dtype=torch.int64, device=dev) if want_steps else None
        if visits is None and want_visits:
            visits = torch.zeros(na * n, dtype=torch.int64, device=dev)
        roots = torch.empty(na * tau * n, dtype=torch.int32, device=dev) if want_roots else None
        depths = torch.empty(na * tau * n, dtype=torch.int32, device=dev) if want_roots else None
        if visits is not None:
            _dev_tensor(visits, torch.int64, na * n, "visits")
        if want_roots:
            _check(lib().fc_sample_usts_forest(self._h, int(seed) & (2**64 - 1), int(tau), int(tree_offset), _ptr(R),
                                               _ptr(C), _ptr(parents), _ptr(roots), _ptr(depths), _ptr(visits),
                                               int(max_steps_per_tree), _ptr(steps), _stream(stream)),
                   "fc_sample_usts_forest")
        elif visits is not None:
            _check(lib().fc_sample_usts_ex(self._h, int(seed) & (2**64 - 1), int(tau), int(tree_offset), _ptr(R),
                                           _ptr(C), _ptr(parents), _ptr(visits), int(max_steps_per_tree),
                                           _ptr(steps), _stream(stream)), "fc_sample_usts_ex")
        else:
            _check(lib().fc_sample_usts(self._h, int(seed) & (2**64 - 1), int(tau), int(tree_offset), _ptr(R),
                                        _ptr(C), _ptr(parents), int(max_steps_per_tree), _ptr(steps),
                                        _stream(stream)), "fc_sample_usts")
        out = {"R": R, "C": C, "visits": visits}
        if want_parents:
            out["parents"] = parents.view(na, tau, n)
        if want_roots:
            out["roots"] = roots.view(na, tau, n)
            out["depths"] = depths.view(na, tau, n)
        if want_steps:
            out["steps"] = steps.view(getattr(self, "num_graphs", 0) or na, tau)
        return out

    def stack_entries(self, seed: int, tree: int, verts, ks, alpha_idx: int = 0, stream=None):
        """fc_stack_entries (diagnostic): vertex chosen by stack entry ks[i] of verts[i]."""
        verts = verts.to(torch.int32).contiguous()
        ks = ks.to(torch.int32).contiguous()
        out = torch.empty_like(verts)
        _check(lib().fc_stack_entries(self._h, alpha_idx, int(seed) & (2**64 - 1), int(tree), verts.numel(),
                                      _ptr(verts), _ptr(ks), _ptr(out), _stream(stream)), "fc_stack_entries")
        return out

    def sampler_stats(self):
        pops = ctypes.c_uint64()
        deps = ctypes.c_uint64()
        _check(lib().fc_sampler_stats(self._h, ctypes.byref(pops), ctypes.byref(deps)), "fc_sampler_stats")
        return int(pops.value), int(deps.value)

    def solve(self, b, alpha_idx: int = 0, x=None, rel_tol: float = 1e-9, max_iter: int = 20000,
              stream=None):
        """fc_solve for b of shape [n] or [m, n] (FP64, CUDA).  Returns (x, iters)."""
        b2 = b.reshape(-1, self.n).contiguous()
        m = b2.shape[0]
        _dev_tensor(b2, torch.float64, m * self.n, "b")
        if x is None:
            x = torch.zeros_like(b2)
        _dev_tensor(x, torch.float64, m * self.n, "x")
        it = ctypes.c_int32()
        _check(lib().fc_solve(self._h, alpha_idx, _ptr(b2), _ptr(x), m, float(rel_tol), int(max_iter),
                              ctypes.byref(it), _stream(stream)), "fc_solve")
        return x.reshape(b.shape), int(it.value)

    def pivot_solve(self, alpha_idx: int = 0, rel_tol: float = 1e-9, max_iter: int = 20000, stream=None):
        """Algorithm 1's pivot solve, x of length n+1 (x[n] = x(u*))."""
        x = torch.empty(self.n + 1, dtype=torch.float64, device=torch.device("cuda", torch.cuda.current_device()))
        it = ctypes.c_int32()
        _check(lib().fc_pivot_solve(self._h, alpha_idx, _ptr(x), float(rel_tol), int(max_iter), ctypes.byref(it),
                                    _stream(stream)), "fc_pivot_solve")
        return x, int(it.value)

    def farness(self, R, tau: int, alpha_idx: int = 0, C=None, g_pred=None, x_pivot=None, stream=None):
        """fc_forest_farness on the alpha slices of R (and C).  Returns diag, farness, closeness."""
        n = self.n
        dev = torch.device("cuda", torch.cuda.current_device())
        Ra = R.view(-1)[alpha_idx * n:(alpha_idx + 1) * n] if R.numel() > n else R
        Ca = None
        if C is not None:
            Ca = C.view(-1)[alpha_idx * n:(alpha_idx + 1) * n] if C.numel() > n else C
        diag = torch.empty(n, dtype=torch.float64, device=dev)
        far = torch.empty(n, dtype=torch.float64, device=dev)
        clo = torch.empty(n, dtype=torch.float64, device=dev)
        if g_pred is not None:
            _dev_tensor(g_pred, torch.float32, n, "g_pred")
        _check(lib().fc_forest_farness(self._h, alpha_idx, _ptr(Ra), _ptr(Ca), _ptr(g_pred), _ptr(x_pivot),
                                       int(tau), _ptr(diag), _ptr(far), _ptr(clo), _stream(stream)),
               "fc_forest_farness")
        return diag, far, clo

    def rb_accumulate(self, parents, acc=None, alpha_idx: int = 0, stream=None):
        """fc_rb_accumulate: add the Rao-Blackwellised values of the trees in
        parents ([T, n] or [n_alpha, T, n] sliced by the caller; int32 CUDA) to acc
        (uint64 as int64 CUDA, allocated zeroed when not given)."""
        n = self.n
        par = parents.reshape(-1, n).contiguous()
        if acc is None:
            acc = torch.zeros(n, dtype=torch.int64, device=par.device)
        _check(lib().fc_rb_accumulate(self._h, int(alpha_idx), _ptr(par), int(par.shape[0]), _ptr(acc),
                                      _stream(stream)), "fc_rb_accumulate")
        return acc

    def rb_diag(self, acc, trees: int, stream=None):
        diag = torch.empty(self.n, dtype=torch.float64, device=acc.device)
        _check(lib().fc_rb_diag(_ptr(acc), int(self.n), int(trees), _ptr(diag), _stream(stream)), "fc_rb_diag")
        return diag

    def visit_diag(self, visits, tau: int, alpha_idx: int = 0, stream=None):
        """fc_visit_diag: diag(Omega) from the visit totals of tau trees."""
        out = torch.empty(self.n, dtype=torch.float64, device=visits.device)
        _check(lib().fc_visit_diag(self._h, alpha_idx, _ptr(visits), int(tau), _ptr(out), _stream(stream)),
               "fc_visit_diag")
        return out

    def farness_from_diag(self, diag, stream=None):
        """fc_farness_from_diag: (farness, closeness) of a diag(Omega) estimate."""
        _dev_tensor(diag, torch.float64, self.n, "diag")
        far = torch.empty_like(diag)
        clo = torch.empty_like(diag)
        _check(lib().fc_farness_from_diag(self._h, _ptr(diag), _ptr(far), _ptr(clo), _stream(stream)),
               "fc_farness_from_diag")
        return far, clo

    def group_closeness(self, k: int, alpha_idx: int = 0, rel_tol: float = 1e-12, stream=None):
        """fc_group_closeness (Algorithm 3): (S, farness) with S the k chosen
        vertices in order (int32 CUDA) and farness[i] = rho(S[:i+1]) (FP64
        CUDA)."""
        dev = torch.device("cuda", torch.cuda.current_device())
        S = torch.empty(int(k), dtype=torch.int32, device=dev)
        far = torch.empty(int(k), dtype=torch.float64, device=dev)
        _check(lib().fc_group_closeness(self._h, int(alpha_idx), int(k), float(rel_tol), _ptr(S), _ptr(far),
                                        _stream(stream)), "fc_group_closeness")
        return S, far

    # ---- learned control variate ----
    def features(self, alpha_idx: int = 0, stream=None):
        X = torch.empty(self.n * 4, dtype=torch.float32, device=torch.device("cuda", torch.cuda.current_device()))
        _check(lib().fc_vertex_features(self._h, alpha_idx, _ptr(X), _stream(stream)), "fc_vertex_features")
        return X.view(self.n, 4)

    def mlp_forward(self, X, params, alpha_idx: int = 0, stream=None):
        out = torch.empty(self.n, dtype=torch.float32, device=X.device)
        _check(lib().fc_mlp_forward(self._h, alpha_idx, _ptr(X.contiguous()), _ptr(params), _ptr(out),
                                    _stream(stream)), "fc_mlp_forward")
        return out

    def mlp_loss_grad(self, X, y, params, alpha_idx: int = 0, stream=None):
        grad = torch.empty_like(params)
        loss = torch.empty(1, dtype=torch.float32, device=params.device)
        _check(lib().fc_mlp_loss_grad(self._h, alpha_idx, _ptr(X.contiguous()), _ptr(y.contiguous()), _ptr(params),
                                      _ptr(grad), _ptr(loss), _stream(stream)), "fc_mlp_loss_grad")
        return loss, grad

    def mlp_loss_grad_acc(self, X, y, params, grad, loss, weight: float, accumulate: bool, alpha_idx: int = 0,
                          stream=None):
        """fc_mlp_loss_grad_acc: grad (and loss) = (accumulate ? old : 0) + weight * this graph's."""
        _check(lib().fc_mlp_loss_grad_acc(self._h, alpha_idx, _ptr(X.contiguous()), _ptr(y.contiguous()),
                                          _ptr(params), float(weight), int(bool(accumulate)), _ptr(grad),
                                          _ptr(loss), _stream(stream)), "fc_mlp_loss_grad_acc")

    def p_root(self, alpha_idx: int = 0, stream=None):
        p = torch.empty(self.n, dtype=torch.float64, device=torch.device("cuda", torch.cuda.current_device()))
        _check(lib().fc_p_root(self._h, alpha_idx, _ptr(p), _stream(stream)), "fc_p_root")
        return p


def top_k(diag, k: int, stream=None):
    _dev_tensor(diag, torch.float64, diag.numel(), "diag")
    out = torch.empty(k, dtype=torch.int32, device=diag.device)
    _check(lib().fc_top_k(_ptr(diag), int(diag.numel()), int(k), _ptr(out), _stream(stream)), "fc_top_k")
    return out


def mlp_param_count() -> int:
    return int(lib().fc_mlp_param_count())


def mlp_adam(params, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
             eps: float = 1e-8, stream=None):
    _check(lib().fc_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.numel(), int(step), float(lr),
                             float(beta1), float(beta2), float(eps), _stream(stream)), "fc_mlp_adam")


def launch_count() -> int:
    """Kernel launches made by libfc.so in this process so far."""
    return int(lib().fc_launch_count())


def tree_roots(parents, want_depth: bool = True, stream=None):
    """fc_tree_roots on parents [T, n] (int32 CUDA): (roots, depth)."""
    T, n = parents.shape[-2], parents.shape[-1]
    par = parents.reshape(T, n).contiguous()
    roots = torch.empty_like(par)
    depth = torch.empty_like(par) if want_depth else None
    _check(lib().fc_tree_roots(_ptr(par), int(n), int(T), _ptr(roots), _ptr(depth), _stream(stream)),
           "fc_tree_roots")
    return roots, depth


def root_counts(roots, queries, counts=None, stream=None):
    """fc_root_counts: counts[q][v] of trees in which v's forest root is queries[q]."""
    T, n = roots.shape
    q = queries.to(torch.int32).contiguous()
    if counts is None:
        counts = torch.zeros(q.numel() * n, dtype=torch.int32, device=roots.device)
    _check(lib().fc_root_counts(_ptr(roots.contiguous()), int(n), int(T), _ptr(q), int(q.numel()), _ptr(counts),
                                _stream(stream)), "fc_root_counts")
    return counts.view(q.numel(), n)


def tau_for(eps: float, delta: float, kappa: float, m: int) -> int:
    return int(lib().fc_tau_for(float(eps), float(delta), float(kappa), int(m)))


def declared_symbols():
    """Entry points declared in include/fc.h (parsed from the header)."""
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fc.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"\b(fc_[a-z0-9_]+)\s*\(", txt)))
