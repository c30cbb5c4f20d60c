"""Python binding of libnesa (the GB300 NESA/EFIE library).

Argument marshalling only: every stage of the product and of the solver runs in the
library's CUDA kernels.  Device vectors are torch tensors (complex128, shape
``[nrhs, N]``, contiguous, on the CUDA device of the context), passed by pointer.
If ``libnesa.so`` is missing or cannot be loaded every call raises; there is no
fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnesa.so")

OK = 0
ERR_INVALID_ARG, ERR_MESH, ERR_CUDA, ERR_OOM, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_NUMERIC = -1, -2, -3, -4, -5, -6, -7
FP64, MIXED = 0, 1
Q_FIXED, Q_AUTO = 0, 1
PART_NEAR, PART_FAR, PART_ALL, PART_MIXED = 1, 2, 3, 4
TRANSLATE_FP32, TRANSLATE_TENSOR = 0, 1
EXPORT_POINT_LEAF, EXPORT_RWG = 1, 2
OP_D, OP_C, OP_OFFSET = 1, 2, 3
MAX_LEVELS = 20


class NesaError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("libnesa status %d (%s)%s" % (status, _status_str(status), (": " + what) if what else ""))


class Mesh(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_triangles", ctypes.c_int64),
                ("vertices", ctypes.c_void_p), ("triangles", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_double), ("n_levels", ctypes.c_int32), ("q_mode", ctypes.c_int32),
                ("q_fixed", ctypes.c_int32), ("precision", ctypes.c_int32), ("q_digits", ctypes.c_double),
                ("rho_eq", ctypes.c_double), ("rho_test", ctypes.c_double), ("pinv_eps", ctypes.c_double),
                ("translate", ctypes.c_int32), ("tile_n", ctypes.c_int32), ("points_per_leaf", ctypes.c_int32),
                ("singular_mode", ctypes.c_int32), ("translation_tables", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("n_unknowns", ctypes.c_int64), ("n_triangles", ctypes.c_int64), ("n_points", ctypes.c_int64),
                ("n_levels", ctypes.c_int32), ("l0", ctypes.c_int32), ("q", ctypes.c_int32 * MAX_LEVELS),
                ("n_boxes", ctypes.c_int64 * MAX_LEVELS), ("n_interactions", ctypes.c_int64 * MAX_LEVELS),
                ("n_offsets", ctypes.c_int64 * MAX_LEVELS), ("near_nnz", ctypes.c_int64),
                ("near_tri_pairs", ctypes.c_int64), ("v_columns", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("build_seconds", ctypes.c_double), ("max_leaf_columns", ctypes.c_int64),
                ("build_split", ctypes.c_double * 4)]

    def as_dict(self):
        nl = self.n_levels
        return dict(n_unknowns=self.n_unknowns, n_triangles=self.n_triangles, n_points=self.n_points,
                    n_levels=nl, l0=self.l0, q=list(self.q[:nl]), n_boxes=list(self.n_boxes[:nl]),
                    n_interactions=list(self.n_interactions[:nl]), n_offsets=list(self.n_offsets[:nl]),
                    near_nnz=self.near_nnz, near_tri_pairs=self.near_tri_pairs, v_columns=self.v_columns,
                    device_bytes=self.device_bytes, build_seconds=self.build_seconds,
                    build_split=dict(zip(("mesh_rwg_host", "tree_lists_device", "near_pattern_host",
                                          "operators_device"), list(self.build_split))),
                    max_leaf_columns=self.max_leaf_columns)


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 5), ("ms", ctypes.c_double * 5), ("flops", ctypes.c_double * 5),
                ("bytes", ctypes.c_double * 5)]


STAGES = ("radiation", "source_transfer", "translation", "near_reception", "translation_tensor_gemm")


class SolveOpts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int32), ("max_iters", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("mixed", ctypes.c_int32), ("max_refine", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("reserved", ctypes.c_int32 * 3)]


class LearnOpts(ctypes.Structure):
    _fields_ = [("samples", ctypes.c_int32), ("steps", ctypes.c_int32), ("lr", ctypes.c_float),
                ("val_iters", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class LearnInfo(ctypes.Structure):
    _fields_ = [("loss_initial", ctypes.c_double), ("loss_final", ctypes.c_double), ("samples", ctypes.c_int32),
                ("steps", ctypes.c_int32), ("seconds", ctypes.c_double), ("val_res_learned", ctypes.c_double),
                ("val_res_base", ctypes.c_double), ("fallback", ctypes.c_int32), ("val_iters", ctypes.c_int32)]


PRECOND_NONE, PRECOND_BLOCK_JACOBI, PRECOND_LEARNED, PRECOND_OVERLAP = 0, 1, 2, 3
SINGULAR_TOUCHING, SINGULAR_SELF = 0, 1
TABLES_AUTO, TABLES_STORED, TABLES_GENERATED = 0, 1, 2
LEARN_PARAMS = 1542


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("matvecs", ctypes.c_int32), ("refinements", ctypes.c_int32), ("fp64_matvecs", ctypes.c_int32),
                ("rel_residual", ctypes.c_double * 64), ("seconds", ctypes.c_double)]

_lib = None


def lib():
    """Load libnesa.so (raises if it is missing: the library has no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libnesa.so not built: run paper_1801_03589_gb300/build.py (or __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "nesa_default_params": (None, [P]),
            "nesa_build": (I, [P, D, P, P]),
            "nesa_plan": (I, [P, D, P, P]),
            "nesa_set_stream": (I, [P, P]),
            "nesa_num_unknowns": (I, [P, P]),
            "nesa_get_info": (I, [P, P]),
            "nesa_matvec": (I, [P, P, P, I]),
            "nesa_matvec_parts": (I, [P, P, P, I, I]),
            "nesa_matvec_host": (I, [P, P, P, I, I]),
            "nesa_rhs_planewave": (I, [P, P, P, I, P]),
            "nesa_export": (I, [P, I, P, ctypes.c_size_t]),
            "nesa_export_op": (I, [P, I, I, I, P, ctypes.c_size_t]),
            "nesa_destroy": (None, [P]),
            "nesa_status_str": (ctypes.c_char_p, [I]),
            "nesa_last_error": (ctypes.c_char_p, []),
            "nesa_profile_enable": (I, [P, I]),
            "nesa_profile_read": (I, [P, P]),
            "nesa_default_solve_opts": (None, [P]),
            "nesa_solve": (I, [P, P, P, I, D, P, P]),
            "nesa_device_status": (I, [P]),
            "nesa_inject_stall": (I, [P, I, ctypes.c_uint32]),
            "nesa_precond_setup": (I, [P]),
            "nesa_precond_apply": (I, [P, I, P, P, I]),
            "nesa_default_learn_opts": (None, [P]),
            "nesa_precond_train": (I, [P, P, I, P, P]),
            "nesa_precond_params": (I, [P, I, P]),
            "nesa_precond_features": (I, [P, P]),
            "nesa_precond_loss_grad": (I, [P, P, P, I, P, P]),
            "nesa_build_batch": (I, [P, I, P, P, P]),
            "nesa_batch_create": (I, [P, I, P, P, P, I, P]),
            "nesa_batch_launch": (I, [P, P]),
            "nesa_batch_kernels": (I, [P, P]),
            "nesa_batch_destroy": (None, [P]),
            "nesa_get_tuning": (I, [P, P, P]),
            "nesa2d_build": (I, [P, I64, I, I, D, P]),
            "nesa2d_set_stream": (I, [P, P]),
            "nesa2d_get_info": (I, [P, P]),
            "nesa2d_matvec": (I, [P, P, P, I, I]),
            "nesa2d_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _status_str(s):
    try:
        return lib().nesa_status_str(s).decode()
    except Exception:  # noqa: BLE001 - only used to format an error
        return "?"


def _check(status):
    if status != OK:
        what = lib().nesa_last_error().decode()
        raise NesaError(status, what)


def default_params(**overrides):
    p = Params()
    lib().nesa_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise TypeError("unknown parameter %s" % k)
        setattr(p, k, v)
    return p


def _dev_ptr(t, n, what):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.complex128 or not t.is_contiguous():
        raise TypeError("%s must be a contiguous complex128 CUDA tensor" % what)
    if t.dim() == 1:
        t = t.view(1, -1)
    if t.shape[-1] != n:
        raise ValueError("%s has %d columns, expected %d" % (what, t.shape[-1], n))
    return t, t.data_ptr(), t.shape[0]


MAX_LEVELS_2D = 32
PART2D_NEAR, PART2D_FAR, PART2D_ALL = 1, 2, 3


class Info2D(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("l0", ctypes.c_int32), ("L", ctypes.c_int32),
                ("q", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n_boxes", ctypes.c_int64 * MAX_LEVELS_2D), ("n_interactions", ctypes.c_int64 * MAX_LEVELS_2D),
                ("n_offsets", ctypes.c_int64 * MAX_LEVELS_2D), ("near_entries", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64)]


class Model2D:
    """The 2D model problem of Sec. 3 (log-kernel potential of charges on a curve):
    one built operator on the current CUDA device (owns its device memory)."""

    def __init__(self, points, P, Q, pinv_eps=0.0):
        x = np.ascontiguousarray(points, dtype=np.float64)
        if x.ndim != 2 or x.shape[1] != 2:
            raise ValueError("points must be [n][2]")
        self.n = x.shape[0]
        h = ctypes.c_void_p()
        _check(lib().nesa2d_build(x.ctypes.data, self.n, int(P), int(Q), float(pinv_eps), ctypes.byref(h)))
        self._h = h

    def info(self):
        i = Info2D()
        _check(lib().nesa2d_get_info(self._h, ctypes.byref(i)))
        levels = range(i.l0, i.L + 1)
        return dict(n_points=i.n_points, l0=i.l0, L=i.L, q=i.q, n_boxes={l: i.n_boxes[l] for l in levels},
                    n_interactions={l: i.n_interactions[l] for l in levels},
                    n_offsets={l: i.n_offsets[l] for l in levels}, near_entries=i.near_entries,
                    device_bytes=i.device_bytes)

    def set_stream(self, stream):
        _check(lib().nesa2d_set_stream(self._h, ctypes.c_void_p(getattr(stream, "cuda_stream", stream))))

    def matvec(self, q, phi=None, parts=PART2D_ALL):
        """phi = K~ q for q a float64 CUDA tensor [n] or [nrhs][n] (rows are vectors)."""
        import torch
        if not isinstance(q, torch.Tensor) or not q.is_cuda or q.dtype != torch.float64 or not q.is_contiguous():
            raise TypeError("q must be a contiguous float64 CUDA tensor")
        if q.shape[-1] != self.n:
            raise ValueError("q has %d columns, expected %d" % (q.shape[-1], self.n))
        nrhs = 1 if q.dim() == 1 else q.shape[0]
        if phi is None:
            phi = torch.empty_like(q)
        _check(lib().nesa2d_matvec(self._h, q.data_ptr(), phi.data_ptr(), nrhs, int(parts)))
        return phi

    def close(self):
        if getattr(self, "_h", None):
            lib().nesa2d_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


class Batch:
    """One CUDA graph holding the products of several operators; launch() runs a pass."""

    def __init__(self, members, xs, ys, parts=PART_ALL):
        n = len(members)
        self._keep = (list(members), list(xs), list(ys))
        ctxs = (ctypes.c_void_p * n)(*[m._h.value for m in members])
        xp = (ctypes.c_void_p * n)()
        yp = (ctypes.c_void_p * n)()
        nr = (ctypes.c_int * n)()
        for i, (m, x, y) in enumerate(zip(members, xs, ys)):
            x, px, nrhs = _dev_ptr(x, m.n, "x")
            y, py, nr2 = _dev_ptr(y, m.n, "y")
            if nr2 != nrhs:
                raise ValueError("x and y differ in nrhs")
            xp[i], yp[i], nr[i] = px, py, nrhs
        h = ctypes.c_void_p()
        _check(lib().nesa_batch_create(ctxs, n, xp, yp, nr, parts, ctypes.byref(h)))
        self._h = h
        k = ctypes.c_int64()
        _check(lib().nesa_batch_kernels(h, ctypes.byref(k)))
        self.kernel_nodes = k.value

    def launch(self, stream=None):
        handle = getattr(stream, "cuda_stream", stream)
        _check(lib().nesa_batch_launch(self._h, ctypes.c_void_p(handle)))

    def close(self):
        if getattr(self, "_h", None):
            lib().nesa_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def plan(vertices, triangles, k, **params):
    """The host part of a build (no device): sizes of the operator nesa_build would make."""
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    t = np.ascontiguousarray(triangles, dtype=np.int32)
    mesh = Mesh(len(v), len(t), v.ctypes.data, t.ctypes.data)
    p = default_params(**params)
    i = Info()
    _check(lib().nesa_plan(ctypes.byref(mesh), float(k), ctypes.byref(p), ctypes.byref(i)))
    return i.as_dict()


def build_batch(meshes, ks, **params):
    """Operators of several meshes built by one nesa_build_batch call: meshes is a list of
    (vertices, triangles), ks their wavenumbers.  Returns a list of Nesa objects."""
    n = len(meshes)
    arrays = [(np.ascontiguousarray(v, dtype=np.float64), np.ascontiguousarray(t, dtype=np.int32))
              for v, t in meshes]
    m = (Mesh * n)(*[Mesh(len(v), len(t), v.ctypes.data, t.ctypes.data) for v, t in arrays])
    k = (ctypes.c_double * n)(*[float(x) for x in ks])
    p = default_params(**params)
    h = (ctypes.c_void_p * n)()
    _check(lib().nesa_build_batch(m, n, k, ctypes.byref(p), h))
    out = []
    for i in range(n):
        g = Nesa.__new__(Nesa)
        g._h = ctypes.c_void_p(h[i])
        g.params = p
        g.k = float(ks[i])
        nn = ctypes.c_int64()
        _check(lib().nesa_num_unknowns(g._h, ctypes.byref(nn)))
        g.n = nn.value
        out.append(g)
    return out


class Nesa:
    """One built operator (owns its device memory)."""

    def __init__(self, vertices, triangles, k, **params):
        v = np.ascontiguousarray(vertices, dtype=np.float64)
        t = np.ascontiguousarray(triangles, dtype=np.int32)
        mesh = Mesh(len(v), len(t), v.ctypes.data, t.ctypes.data)
        self.params = default_params(**params)
        h = ctypes.c_void_p()
        _check(lib().nesa_build(ctypes.byref(mesh), float(k), ctypes.byref(self.params), ctypes.byref(h)))
        self._h = h
        self.k = float(k)
        n = ctypes.c_int64()
        _check(lib().nesa_num_unknowns(h, ctypes.byref(n)))
        self.n = n.value

    def close(self):
        if getattr(self, "_h", None):
            lib().nesa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def info(self):
        i = Info()
        _check(lib().nesa_get_info(self._h, ctypes.byref(i)))
        return i.as_dict()

    def set_stream(self, stream):
        """Order the context's device work on a torch.cuda.Stream (or a raw handle)."""
        handle = getattr(stream, "cuda_stream", stream)
        _check(lib().nesa_set_stream(self._h, ctypes.c_void_p(handle)))

    def matvec(self, x, y=None, parts=PART_ALL):
        """y = Z~ x for x of shape [nrhs, N] (complex128, CUDA).  Asynchronous."""
        import torch
        x, px, nrhs = _dev_ptr(x, self.n, "x")
        if y is None:
            y = torch.empty_like(x)
        y, py, nr2 = _dev_ptr(y, self.n, "y")
        if nr2 != nrhs:
            raise ValueError("x and y differ in nrhs")
        _check(lib().nesa_matvec_parts(self._h, px, py, nrhs, parts))
        return y

    def matvec_host(self, x, parts=PART_ALL):
        """End to end from host memory: x numpy or CPU tensor [nrhs, N] complex128."""
        xa = np.ascontiguousarray(np.atleast_2d(np.asarray(x)), dtype=np.complex128)
        y = np.empty_like(xa)
        _check(lib().nesa_matvec_host(self._h, xa.ctypes.data, y.ctypes.data, xa.shape[0], parts))
        return y

    def matvec_host_ptr(self, x_ptr, y_ptr, nrhs, parts=PART_ALL):
        """End to end product between two host buffers given by address (e.g. pinned tensors)."""
        _check(lib().nesa_matvec_host(self._h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), int(nrhs), parts))

    def rhs_planewave(self, khat, pol, out=None):
        import torch
        kh = np.ascontiguousarray(np.atleast_2d(khat), dtype=np.float64)
        pl = np.ascontiguousarray(np.atleast_2d(pol), dtype=np.complex128)
        nrhs = kh.shape[0]
        if out is None:
            out = torch.empty((nrhs, self.n), dtype=torch.complex128, device="cuda")
        out, po, nr2 = _dev_ptr(out, self.n, "out")
        if nr2 != nrhs or pl.shape != (nrhs, 3):
            raise ValueError("khat, pol and out disagree in nrhs")
        _check(lib().nesa_rhs_planewave(self._h, kh.ctypes.data, pl.ctypes.data, nrhs, po))
        return out

    # ------------------------------------------------------------ preconditioners
    def precond_apply(self, r, kind=PRECOND_BLOCK_JACOBI):
        import torch
        r, pr, nrhs = _dev_ptr(r, self.n, "r")
        z = torch.empty_like(r)
        _check(lib().nesa_precond_apply(self._h, kind, pr, z.data_ptr(), nrhs))
        return z

    def precond_train(self, b, samples=48, steps=300, lr=3e-3, val_iters=100):
        b, pb, nrhs = _dev_ptr(b, self.n, "b")
        o = LearnOpts()
        lib().nesa_default_learn_opts(ctypes.byref(o))
        o.samples, o.steps, o.lr, o.val_iters = int(samples), int(steps), float(lr), int(val_iters)
        i = LearnInfo()
        _check(lib().nesa_precond_train(self._h, pb, nrhs, ctypes.byref(o), ctypes.byref(i)))
        return dict(loss_initial=i.loss_initial, loss_final=i.loss_final, samples=i.samples, steps=i.steps,
                    seconds=i.seconds, val_res_learned=i.val_res_learned, val_res_base=i.val_res_base,
                    fallback=i.fallback, val_iters=i.val_iters)

    def precond_params(self, values=None):
        """Get the learned weights (values None) or set them (marks the network trained)."""
        a = np.zeros(LEARN_PARAMS, np.float32) if values is None else np.ascontiguousarray(values, np.float32)
        _check(lib().nesa_precond_params(self._h, 0 if values is None else 1, a.ctypes.data))
        return a

    def precond_features(self):
        a = np.zeros((self.n, 8), np.float32)
        _check(lib().nesa_precond_features(self._h, a.ctypes.data))
        return a

    def precond_loss_grad(self, u, v):
        u, pu, ns = _dev_ptr(u, self.n, "u")
        v, pv, ns2 = _dev_ptr(v, self.n, "v")
        if ns != ns2:
            raise ValueError("u and v differ in sample count")
        loss = ctypes.c_double()
        g = np.zeros(LEARN_PARAMS, np.float32)
        _check(lib().nesa_precond_loss_grad(self._h, pu, pv, ns, ctypes.byref(loss), g.ctypes.data))
        return loss.value, g

    def solve(self, b, tol, x=None, restart=50, max_iters=1000, check=True, mixed=False, max_refine=10,
              inner_tol=3e-3, precond=PRECOND_NONE):
        """Restarted GMRES on the device for Z~ x = b (b: [nrhs, N] complex128 CUDA).
        mixed=True: FP64 iterative refinement around GMRES on the low-precision product.
        Returns (x, info dict).  With check=False a non-converged solve returns instead
        of raising (info['status'] holds the library status)."""
        import torch
        b, pb, nrhs = _dev_ptr(b, self.n, "b")
        if x is None:
            x = torch.empty_like(b)
        x, px, nr2 = _dev_ptr(x, self.n, "x")
        o = SolveOpts()
        lib().nesa_default_solve_opts(ctypes.byref(o))
        o.restart, o.max_iters = int(restart), int(max_iters)
        o.mixed, o.max_refine, o.inner_tol = int(bool(mixed)), int(max_refine), float(inner_tol)
        o.precond = int(precond)
        i = SolveInfo()
        st = lib().nesa_solve(self._h, pb, px, nrhs, float(tol), ctypes.byref(o), ctypes.byref(i))
        info = dict(status=st, iterations=i.iterations, restarts=i.restarts, converged=i.converged,
                    matvecs=i.matvecs, refinements=i.refinements, fp64_matvecs=i.fp64_matvecs,
                    rel_residual=list(i.rel_residual[:nrhs]), seconds=i.seconds)
        if check and st != OK:
            raise NesaError(st, str(info))
        return x, info

    def device_status(self):
        """Status of the context's kernels since the last call (OK or ERR_TIMEOUT); clears it."""
        return lib().nesa_device_status(self._h)

    def inject_stall(self, stall, wait_limit=0):
        """Failure-detection hook: stall the tensor GEMM producers so its bounded waits
        (wait_limit iterations; 0 = default) run out at the next mixed product."""
        _check(lib().nesa_inject_stall(self._h, int(stall), int(wait_limit)))

    def profile_enable(self, on=True):
        _check(lib().nesa_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        """Per-stage totals since profile_enable: launches, device ms, algorithmic flops and bytes."""
        p = Profile()
        _check(lib().nesa_profile_read(self._h, ctypes.byref(p)))
        return {name: dict(launches=p.launches[i], ms=p.ms[i], flops=p.flops[i], bytes=p.bytes[i])
                for i, name in enumerate(STAGES)}

    def tuning(self):
        """Tile width chosen per level by the autotuner and the measured times (ms) for
        widths 64, 128, 256."""
        tn = (ctypes.c_int32 * MAX_LEVELS)()
        ms = (ctypes.c_float * (3 * MAX_LEVELS))()
        _check(lib().nesa_get_tuning(self._h, tn, ms))
        return {l: dict(tile_n=tn[l], ms=list(ms[3 * l:3 * l + 3])) for l in range(MAX_LEVELS) if tn[l]}

    def export_point_leaf(self):
        a = np.empty((self.info()["n_points"], 3), np.int32)
        _check(lib().nesa_export(self._h, EXPORT_POINT_LEAF, a.ctypes.data, a.nbytes))
        return a

    def export_rwg(self):
        a = np.empty((self.n, 4), np.int32)
        _check(lib().nesa_export(self._h, EXPORT_RWG, a.ctypes.data, a.nbytes))
        return a

    def export_offset(self, level, slot):
        """Offset (target - source, in boxes) of translation slot `slot` at `level`."""
        a = np.empty(3, np.int32)
        _check(lib().nesa_export_op(self._h, OP_OFFSET, level, slot, a.ctypes.data, a.nbytes))
        return a

    def export_D(self, level, slot):
        """D_l of translation slot `slot` (complex128, Q_l x Q_l)."""
        q = self.info()["q"][level]
        a = np.empty((q, q), np.complex128, order="F")
        _check(lib().nesa_export_op(self._h, OP_D, level, slot, a.ctypes.data, a.nbytes))
        return a

    def export_C(self, level, octant):
        """C_l of the child octant (bits x | y << 1 | z << 2; complex128, Q_{l-1} x Q_l)."""
        q = self.info()["q"]
        a = np.empty((q[level - 1], q[level]), np.complex128, order="F")
        _check(lib().nesa_export_op(self._h, OP_C, level, octant, a.ctypes.data, a.nbytes))
        return a
