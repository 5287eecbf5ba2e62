"""Thin Python binding of libhho (argument marshalling only).

Every computation runs in the CUDA library; this module converts meshes and
torch CUDA tensors into the plain pointers and sizes of the C ABI declared in
``include/hho.h``.  Importing it loads ``libhho.so`` from the package
directory and raises if the library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhho.so")

HHO_OK = 0
STATUS = {0: "HHO_OK", 1: "HHO_ERR_ARG", 2: "HHO_ERR_MESH", 3: "HHO_ERR_CUDA", 4: "HHO_ERR_NOMEM",
          5: "HHO_ERR_SINGULAR", 6: "HHO_ERR_NOT_CONVERGED", 7: "HHO_ERR_TIMEOUT", 8: "HHO_ERR_STATE",
          9: "HHO_ERR_UNSUPPORTED"}
COND = {"v": 0, "vp": 1, "hp": 2, "unc": 3, "dg": 4}
NODES = {"elem": 0, "face": 1}

# every entry point declared in include/hho.h
SYMBOLS = ["hho_setup", "hho_ndof", "hho_quad_nodes", "hho_assemble", "hho_assemble_noalloc", "pmg_setup", "pmg_vcycle", "hho_spmv", "hho_spmv_f32",
           "hho_solve", "hho_recover", "hho_errors", "hho_get_element_schur", "hho_get_level_coo",
           "hho_set_element_schur", "hho_launch_count", "hho_coarse_info", "hho_set_option", "hho_destroy",
           "hho_last_error", "hho_set_batch", "hho_solve_batch", "hho_autotune", "hho_mlp_init", "hho_mlp_dims",
           "hho_mlp_weights", "hho_mlp_features", "hho_mlp_apply", "hho_mlp_generate", "hho_mlp_train", "hho_mlp_grads",
           "hho_ilu_apply"]


class HHOError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Mesh(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_vert", C.c_int64), ("xyz", C.POINTER(C.c_double)),
                ("n_elem", C.c_int64), ("elem_face_ptr", C.POINTER(C.c_int64)), ("elem_face", C.POINTER(C.c_int64)),
                ("n_face", C.c_int64), ("face_vert_ptr", C.POINTER(C.c_int64)), ("face_vert", C.POINTER(C.c_int64)),
                ("face_elem", C.POINTER(C.c_int64)), ("face_bc", C.POINTER(C.c_int8))]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("coarse_iterations", C.c_int32), ("rel_residual", C.c_double),
                ("solve_ms", C.c_double), ("status", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load libhho.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libhho.so not found at {path}; build it with paper_2009_13840_gb300.build.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    sig = {
        "hho_setup": (C.c_int, [C.POINTER(_Mesh), C.c_int, C.c_int, P, C.POINTER(P)]),
        "hho_ndof": (C.c_int, [P, C.c_int, C.POINTER(C.c_int64)]),
        "hho_quad_nodes": (C.c_int, [P, C.c_int, C.POINTER(C.c_int64), P, P]),
        "hho_assemble": (C.c_int, [P, P, P, P, P]),
        "hho_assemble_noalloc": (C.c_int, [P, P, P, P, P]),
        "pmg_setup": (C.c_int, [P, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int]),
        "pmg_vcycle": (C.c_int, [P, P, P]),
        "hho_spmv": (C.c_int, [P, C.c_int, P, P]),
        "hho_spmv_f32": (C.c_int, [P, C.c_int, P, P]),
        "hho_solve": (C.c_int, [P, C.c_double, C.c_int, C.c_int, P, C.POINTER(SolveInfo)]),
        "hho_recover": (C.c_int, [P, P, P]),
        "hho_errors": (C.c_int, [P, P, P, P, P, C.POINTER(C.c_double)]),
        "hho_get_element_schur": (C.c_int, [P, P, C.POINTER(C.c_int64)]),
        "hho_get_level_coo": (C.c_int, [P, C.c_int, P, P, P, C.POINTER(C.c_int64)]),
        "hho_set_element_schur": (C.c_int, [P, P]),
        "hho_launch_count": (C.c_int, [P, C.POINTER(C.c_int64)]),
        "hho_coarse_info": (C.c_int, [P, C.POINTER(C.c_int64)]),
        "hho_set_option": (C.c_int, [P, C.c_char_p, C.c_double]),
        "hho_destroy": (C.c_int, [P]),
        "hho_last_error": (C.c_char_p, [P]),
        "hho_set_batch": (C.c_int, [P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "hho_solve_batch": (C.c_int, [P, C.c_double, C.c_int, C.c_int, P, C.POINTER(C.c_int32),
                                      C.POINTER(C.c_double), C.POINTER(SolveInfo)]),
        "hho_autotune": (C.c_int, [P, C.c_int, C.POINTER(C.c_double)]),
        "hho_mlp_init": (C.c_int, [P, C.c_int, C.c_uint64]),
        "hho_mlp_dims": (C.c_int, [P, C.POINTER(C.c_int32)]),
        "hho_mlp_weights": (C.c_int, [P, C.c_int] + [C.POINTER(C.c_double)] * 4),
        "hho_mlp_features": (C.c_int, [P, P, P, P]),
        "hho_mlp_apply": (C.c_int, [P, P, P]),
        "hho_mlp_generate": (C.c_int, [P, C.c_int, C.c_uint64, C.c_int, C.POINTER(C.c_int64)]),
        "hho_mlp_train": (C.c_int, [P, C.c_int, C.c_int, C.c_double, C.c_uint64, C.POINTER(C.c_double)]),
        "hho_mlp_grads": (C.c_int, [P, P, P, C.c_int, C.POINTER(C.c_double)] + [C.POINTER(C.c_double)] * 4),
        "hho_ilu_apply": (C.c_int, [P, C.c_int, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t):
    """Device pointer of a contiguous torch CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _vec(t, dtype, n, what):
    """Device pointer of a contiguous CUDA tensor of `dtype` holding at least
    n values: the library reads and writes exactly n, so a smaller or
    mistyped buffer is refused here rather than overrun on the device."""
    if t is None:
        raise ValueError(f"{what}: a tensor is required")
    if t.dtype != dtype:
        raise TypeError(f"{what}: expected {dtype}, got {t.dtype}")
    if t.numel() < n:
        raise ValueError(f"{what}: expected {n} values, got {t.numel()}")
    return _ptr(t)


@dataclass
class MeshArrays:
    """Host arrays of a mesh in the layout of the C ABI."""
    dim: int
    xyz: np.ndarray
    elem_face_ptr: np.ndarray
    elem_face: np.ndarray
    face_vert_ptr: np.ndarray
    face_vert: np.ndarray
    face_elem: np.ndarray
    face_bc: np.ndarray

    @classmethod
    def from_mesh(cls, m):
        return cls(m.dim, np.ascontiguousarray(m.xyz, np.float64), np.ascontiguousarray(m.elem_face_ptr, np.int64),
                   np.ascontiguousarray(m.elem_face, np.int64), np.ascontiguousarray(m.face_vert_ptr, np.int64),
                   np.ascontiguousarray(m.face_vert, np.int64), np.ascontiguousarray(m.face_elem, np.int64).ravel(),
                   np.ascontiguousarray(m.face_bc, np.int8))


class Context:
    """One discretisation (mesh, degree, condensation) on the current CUDA device."""

    def __init__(self, mesh, k: int, cond: str = "vp", stream=None):
        import torch
        self._torch = torch
        self.lib = load()
        self.mesh = mesh
        self.k = k
        self.cond = cond
        a = MeshArrays.from_mesh(mesh)
        self._keep = a
        cm = _Mesh(a.dim, a.xyz.shape[0], a.xyz.ctypes.data_as(C.POINTER(C.c_double)),
                   a.elem_face_ptr.shape[0] - 1, a.elem_face_ptr.ctypes.data_as(C.POINTER(C.c_int64)),
                   a.elem_face.ctypes.data_as(C.POINTER(C.c_int64)), a.face_vert_ptr.shape[0] - 1,
                   a.face_vert_ptr.ctypes.data_as(C.POINTER(C.c_int64)), a.face_vert.ctypes.data_as(C.POINTER(C.c_int64)),
                   a.face_elem.ctypes.data_as(C.POINTER(C.c_int64)), a.face_bc.ctypes.data_as(C.POINTER(C.c_int8)))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = C.c_void_p()
        st = self.lib.hho_setup(C.byref(cm), k, COND[cond], C.c_void_p(self.stream.cuda_stream), C.byref(self.h))
        self._check(st)
        self.dim = mesh.dim

    # --- plumbing ---
    def _check(self, st):
        if st != HHO_OK:
            msg = self.lib.hho_last_error(self.h).decode() if self.h else ""
            raise HHOError(st, msg)

    def close(self):
        if self.h:
            self.lib.hho_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, *shape):
        return self._torch.empty(*shape, dtype=self._torch.float64, device="cuda")

    # --- API ---
    def ndof(self, level: int = 0) -> int:
        n = C.c_int64()
        self._check(self.lib.hho_ndof(self.h, level, C.byref(n)))
        return n.value

    def quad_nodes(self, which: str):
        n = C.c_int64()
        self._check(self.lib.hho_quad_nodes(self.h, NODES[which], C.byref(n), None, None))
        xyz = self._empty(n.value, self.dim)
        nrm = self._empty(n.value, self.dim) if which == "face" else None
        self._check(self.lib.hho_quad_nodes(self.h, NODES[which], C.byref(n), _ptr(xyz), _ptr(nrm)))
        return (xyz, nrm) if which == "face" else xyz

    def _node_count(self, which):
        n = C.c_int64()
        self._check(self.lib.hho_quad_nodes(self.h, NODES[which], C.byref(n), None, None))
        return n.value

    def _data_ptrs(self, f, gD, gN, rhs_out):
        f64 = self._torch.float64
        ne, nf = self._node_count("elem") * self.dim, self._node_count("face") * self.dim
        return (_vec(f, f64, ne, "f"), _vec(gD, f64, nf, "gD"), _vec(gN, f64, nf, "gN"),
                None if rhs_out is None else _vec(rhs_out, f64, self.ndof(0), "rhs_out"))

    def assemble(self, f, gD, gN, rhs_out=None):
        self._check(self.lib.hho_assemble(self.h, *self._data_ptrs(f, gD, gN, rhs_out)))

    def assemble_noalloc(self, f, gD, gN, rhs_out=None):
        """hho_assemble_noalloc: the library only enqueues the work on the
        context's stream.  The tensors are marked as in use on that stream (so
        torch's caching allocator keeps their memory until the kernels have
        run, even if the caller drops them at once) and the caller's current
        stream is ordered after the work, so that rhs_out is ready for it.
        Neither step allocates device memory."""
        ptrs = self._data_ptrs(f, gD, gN, rhs_out)
        self._check(self.lib.hho_assemble_noalloc(self.h, *ptrs))
        cur = self._torch.cuda.current_stream()
        if cur != self.stream:
            for t in (f, gD, gN, rhs_out):
                if t is not None:
                    t.record_stream(self.stream)
            cur.wait_stream(self.stream)

    def pmg_setup(self, degrees, smooth_its: int = 2, prec="fp64"):
        prec = {"fp64": 0, "fp32": 1, 0: 0, 1: 1}[prec]
        arr = (C.c_int * len(degrees))(*degrees)
        self._check(self.lib.pmg_setup(self.h, len(degrees), arr, prec, smooth_its))
        self.degrees = list(degrees)

    def vcycle(self, r, z):
        n, f64 = self.ndof(0), self._torch.float64
        pr, pz = _vec(r, f64, n, "r"), _vec(z, f64, n, "z")
        if pr.value == pz.value:
            raise ValueError("vcycle: r and z must be different buffers")
        self._check(self.lib.pmg_vcycle(self.h, pr, pz))

    def spmv(self, level, x, y):
        n, f64 = self.ndof(level), self._torch.float64
        self._check(self.lib.hho_spmv(self.h, level, _vec(x, f64, n, "x"), _vec(y, f64, n, "y")))

    def spmv_f32(self, level, x, y):
        n, f32 = self.ndof(level), self._torch.float32
        self._check(self.lib.hho_spmv_f32(self.h, level, _vec(x, f32, n, "x"), _vec(y, f32, n, "y")))

    def solve(self, x, rtol=1e-8, maxit=1000, restart=50, raise_on_fail=True):
        info = SolveInfo()
        px = _vec(x, self._torch.float64, self.ndof(0), "x")
        st = self.lib.hho_solve(self.h, rtol, maxit, restart, px, C.byref(info))
        if raise_on_fail:
            self._check(st)
        return info.as_dict()

    def set_batch(self, face_off, elem_off):
        """Declare the mesh a disjoint union of problems (offsets of n_prob + 1 entries)."""
        fo = np.ascontiguousarray(face_off, dtype=np.int64)
        eo = np.ascontiguousarray(elem_off, dtype=np.int64)
        if fo.shape != eo.shape or fo.ndim != 1:
            raise ValueError("face_off and elem_off must be 1-D of the same length")
        self._check(self.lib.hho_set_batch(self.h, int(fo.size - 1), fo.ctypes.data_as(C.POINTER(C.c_int64)),
                                           eo.ctypes.data_as(C.POINTER(C.c_int64))))
        self.n_prob = int(fo.size - 1)

    def solve_batch(self, x, rtol=1e-8, maxit=1000, restart=50, raise_on_fail=True):
        """One FGMRES per problem of the declared batch; returns (info, iterations, relative residuals)."""
        info = SolveInfo()
        its = np.zeros(self.n_prob, dtype=np.int32)
        rr = np.zeros(self.n_prob, dtype=np.float64)
        st = self.lib.hho_solve_batch(self.h, rtol, maxit, restart, _vec(x, self._torch.float64, self.ndof(0), "x"),
                                      its.ctypes.data_as(C.POINTER(C.c_int32)),
                                      rr.ctypes.data_as(C.POINTER(C.c_double)), C.byref(info))
        if raise_on_fail:
            self._check(st)
        return info.as_dict(), its, rr

    def autotune(self, reps=5):
        """Time the operator-kernel variants (and batch tile sizes) and keep the fastest."""
        out = (C.c_double * 3)()
        self._check(self.lib.hho_autotune(self.h, int(reps), out))
        return dict(spmv_rows=int(out[0]), spmv_grid=int(out[1]), tile_rows=int(out[2]))

    def ilu_apply(self, level, v, z):
        """z = (L U)^{-1} v with the level's block ILU(0) factors (FP64)."""
        n, f64 = self.ndof(int(level)), self._torch.float64
        self._check(self.lib.hho_ilu_apply(self.h, int(level), _vec(v, f64, n, "v"), _vec(z, f64, n, "z")))

    # ---- learned smoother ----
    def mlp_init(self, hidden=128, seed=0):
        self._check(self.lib.hho_mlp_init(self.h, int(hidden), int(seed)))
        return self.mlp_dims()

    def mlp_dims(self):
        d = (C.c_int32 * 4)()
        self._check(self.lib.hho_mlp_dims(self.h, d))
        return dict(din=d[0], hid=d[1], dout=d[2], raw=d[3])

    def mlp_weights(self, new=None):
        """Current FP32 master parameters (dict of numpy arrays), or set them from `new`."""
        d = self.mlp_dims()
        shapes = dict(W1=(d["din"], d["hid"]), b1=(d["hid"],), W2=(d["hid"], d["dout"]), b2=(d["dout"],))
        arrs = {k: np.zeros(v) if new is None else np.ascontiguousarray(new[k], dtype=np.float64).reshape(v)
                for k, v in shapes.items()}
        ptrs = [arrs[k].ctypes.data_as(C.POINTER(C.c_double)) for k in ("W1", "b1", "W2", "b2")]
        self._check(self.lib.hho_mlp_weights(self.h, 0 if new is None else 1, *ptrs))
        return arrs

    def mlp_features(self, r):
        d = self.mlp_dims()
        nf = self.mesh.n_face
        X = self._torch.empty((nf, d["din"]), dtype=self._torch.float32, device="cuda")
        s = self._torch.empty(nf, dtype=self._torch.float32, device="cuda")
        self._check(self.lib.hho_mlp_features(self.h, _ptr(r), _ptr(X), _ptr(s)))
        return X, s

    def mlp_apply(self, v, z):
        """z[face rows] += the learned correction of v (hho_mlp_apply)."""
        n, f64 = self.ndof(0), self._torch.float64
        pv, pz = _vec(v, f64, n, "v"), _vec(z, f64, n, "z")
        self._check(self.lib.hho_mlp_apply(self.h, pv, pz))

    def mlp_generate(self, n_vec, seed=0, kind=2):
        n = C.c_int64()
        self._check(self.lib.hho_mlp_generate(self.h, int(n_vec), int(seed), int(kind), C.byref(n)))
        return n.value

    def mlp_train(self, steps, batch=4096, lr=1e-3, seed=0):
        loss = np.zeros(steps)
        self._check(self.lib.hho_mlp_train(self.h, int(steps), int(batch), float(lr), int(seed),
                                           loss.ctypes.data_as(C.POINTER(C.c_double))))
        return loss

    def mlp_grads(self, X, T):
        d = self.mlp_dims()
        g = dict(W1=np.zeros((d["din"], d["hid"])), b1=np.zeros(d["hid"]), W2=np.zeros((d["hid"], d["dout"])),
                 b2=np.zeros(d["dout"]))
        loss = C.c_double()
        ptrs = [g[k].ctypes.data_as(C.POINTER(C.c_double)) for k in ("W1", "b1", "W2", "b2")]
        self._check(self.lib.hho_mlp_grads(self.h, _ptr(X), _ptr(T), int(X.shape[0]), C.byref(loss), *ptrs))
        return loss.value, g

    def recover(self, x):
        n_loc = self.local_size()
        out = self._empty(n_loc)
        self._check(self.lib.hho_recover(self.h, _vec(x, self._torch.float64, self.ndof(0), "x"), _ptr(out)))
        return out

    def local_size(self):
        """Length of hho_recover's output: per element [U_T | U_F.. | P_T] (Scheme 1),
        [U_T | U_F.. | P_T | P_F..] with U_T of degree k+1 (HHO-hp), [u_T | p_T] (DG)."""
        d, k = self.dim, self.k
        nE = _dimP(d, k)
        nF = _dimP(d - 1, k)
        N = np.diff(self.mesh.elem_face_ptr)
        if self.cond == "dg":
            return int(len(N) * (d + 1) * nE)
        if self.cond == "hp":
            return int(np.sum(d * _dimP(d, k + 1) + N * d * nF + nE + N * nF))
        return int(np.sum(d * nE + N * d * nF + nE))

    def errors(self, local, u, gu, p):
        out = (C.c_double * 4)()
        self._check(self.lib.hho_errors(self.h, _ptr(local), _ptr(u), _ptr(gu), _ptr(p), out))
        return dict(u=out[0], gu=out[1], p=out[2], div=out[3])

    def set_option(self, key: str, value: float):
        self._check(self.lib.hho_set_option(self.h, key.encode(), float(value)))

    def coarse_info(self) -> dict:
        a = (C.c_int64 * 4)()
        self._check(self.lib.hho_coarse_info(self.h, a))
        return {"kind": ["dense", "twolevel", "multifrontal"][a[0]], "values_per_solve": int(a[1]),
                "launches_per_solve": int(a[2]), "factor_values": int(a[3])}

    def launch_count(self) -> int:
        n = C.c_int64()
        self._check(self.lib.hho_launch_count(self.h, C.byref(n)))
        return n.value

    def element_schur(self) -> np.ndarray:
        n = C.c_int64()
        self._check(self.lib.hho_get_element_schur(self.h, None, C.byref(n)))
        buf = np.empty(n.value, dtype=np.float64)
        self._check(self.lib.hho_get_element_schur(self.h, buf.ctypes.data_as(C.c_void_p), C.byref(n)))
        return buf

    def set_element_schur(self, values: np.ndarray):
        v = np.ascontiguousarray(values, np.float64)
        self._check(self.lib.hho_set_element_schur(self.h, v.ctypes.data_as(C.c_void_p)))

    def level_coo(self, level: int):
        n = C.c_int64()
        self._check(self.lib.hho_get_level_coo(self.h, level, None, None, None, C.byref(n)))
        rows = np.empty(n.value, np.int64)
        cols = np.empty(n.value, np.int64)
        vals = np.empty(n.value, np.float64)
        self._check(self.lib.hho_get_level_coo(self.h, level, rows.ctypes.data_as(C.c_void_p),
                                               cols.ctypes.data_as(C.c_void_p), vals.ctypes.data_as(C.c_void_p),
                                               C.byref(n)))
        return rows, cols, vals


def _dimP(nv, deg):
    if nv == 1:
        return deg + 1
    if nv == 2:
        return (deg + 1) * (deg + 2) // 2
    return (deg + 1) * (deg + 2) * (deg + 3) // 6


def _chunked(fn, *arrays, chunk=1 << 20):
    """fn over row chunks of the arrays on a thread pool (numpy releases the
    GIL in its elementwise kernels), concatenated in order."""
    from concurrent.futures import ThreadPoolExecutor
    n = arrays[0].shape[0]
    if n <= chunk:
        return np.ascontiguousarray(fn(*arrays))
    parts = [(i, min(i + chunk, n)) for i in range(0, n, chunk)]
    with ThreadPoolExecutor(max_workers=min(len(parts), os.cpu_count() or 1)) as ex:
        res = list(ex.map(lambda ab: fn(*[a[ab[0]:ab[1]] for a in arrays]), parts))
    return np.ascontiguousarray(np.concatenate(res))


def data_arrays(ctx: Context, field):
    """Evaluate a manufactured field at the library's data nodes; returns CUDA tensors (f, gD, gN).
    (Input preparation on the host: the field is the caller's data, not part of the method.)"""
    import torch
    xe = ctx.quad_nodes("elem").cpu().numpy()
    xf, nf = ctx.quad_nodes("face")
    xf, nf = xf.cpu().numpy(), nf.cpu().numpy()
    f = torch.from_numpy(_chunked(field.f, xe)).cuda()
    gD = torch.from_numpy(_chunked(field.u, xf)).cuda()
    gN = torch.from_numpy(_chunked(field.g_neumann, xf, nf)).cuda()
    return f, gD, gN
