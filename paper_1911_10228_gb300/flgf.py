"""Python binding of the CUDA FLGF library (``libflgf.so``, C ABI in include/flgf.h).

Argument marshalling only: every step of the solver runs in the library's
sm_103a kernels.  PyTorch provides device memory for caller buffers and the
CUDA stream the library enqueues on.  There is no CPU fallback: constructing
a :class:`Context` without the built library or without a GPU raises.

Streams: each Context owns a dedicated ``torch.cuda.Stream`` (needed for
CUDA-graph capture).  Calls that read caller tensors first make the library
stream wait for the caller's current stream; calls that write caller tensors
make the caller's current stream wait for the library stream afterwards.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

FLGF_FP64, FLGF_FP32 = 0, 1
FLGF_HOST, FLGF_DEVICE = 0, 1
OPT_CORRECTION, OPT_GRAPH, OPT_TIMING, OPT_COMPENSATED, OPT_FAULT_HALO = 1, 2, 3, 4, 5
CTX_LIST_PCT, CTX_TILE, CTX_FAIL_ALLOC = 1, 2, 3
# error codes of include/flgf.h
FLGF_EINVAL, FLGF_ENOMEM, FLGF_ECUDA, FLGF_EMESH, FLGF_ESTATE, FLGF_EDEVICE = -1, -2, -3, -4, -5, -6
STAGES = ("coarsen", "anterpolation", "fft_forward", "spectrum_mac", "fft_inverse", "interpolation", "multires")

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_i32_p = ctypes.POINTER(ctypes.c_int32)
_c_i64_p = ctypes.POINTER(ctypes.c_int64)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)


class FLGFError(RuntimeError):
    """A library call failed; ``code`` is its FLGF_E* return code."""

    def __init__(self, msg: str, code: int = 0):
        super().__init__(msg)
        self.code = code


class _Opts(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("n_interp", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_oct_levels", ctypes.c_int), ("table_radius", ctypes.c_int), ("asym_radius", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


# Exported symbols and their prototypes (restype, argtypes).
PROTOTYPES = {
    "flgf_default_opts": (None, [ctypes.POINTER(_Opts)]),
    "flgf_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_Opts)]),
    "flgf_destroy": (None, [ctypes.c_void_p]),
    "flgf_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "flgf_lgf_eval": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_i32_p, _c_dbl_p]),
    "flgf_kernel_spectrum": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            _c_dbl_p]),
    "flgf_blockset_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_int_p, _c_int_p, _c_i32_p, _c_dbl_p,
                                            ctypes.POINTER(ctypes.c_void_p)]),
    "flgf_blockset_create_masked": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_int_p, _c_int_p, _c_i32_p,
                                                   _c_dbl_p, ctypes.POINTER(ctypes.c_uint8),
                                                   ctypes.POINTER(ctypes.c_void_p)]),
    "flgf_blockset_create_vector": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _c_int_p, _c_i32_p,
                                                   ctypes.c_double, ctypes.POINTER(ctypes.c_void_p)]),
    "flgf_blockset_destroy": (None, [ctypes.c_void_p]),
    "flgf_blockset_dof": (ctypes.c_int64, [ctypes.c_void_p]),
    "flgf_load_source": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "flgf_solve": (ctypes.c_int, [ctypes.c_void_p]),
    "flgf_get_potential": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "flgf_laplacian": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int]),
    "flgf_set_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "flgf_ctx_set_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "flgf_stage_times": (ctypes.c_int, [ctypes.c_void_p, _c_dbl_p, ctypes.c_int, _c_int_p, ctypes.c_int]),
    "flgf_work_counts": (ctypes.c_int, [ctypes.c_void_p, _c_i64_p, _c_i64_p, _c_i64_p, _c_i64_p]),
    "flgf_launch_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "flgf_load_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "flgf_solve_adjoint": (ctypes.c_int, [ctypes.c_void_p]),
    "flgf_get_gradient": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "flgf_refine_level": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_double,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "flgf_convolve_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_i32_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_double]),
}

_LIB = None


def load_library(path: str | None = None):
    """Load libflgf.so (built in-tree by ``build.build()``) and declare prototypes."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.LIB
    if not os.path.exists(path):
        raise FLGFError(f"{path} is missing: build the CUDA library first (__graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Context:
    """Block size N, interpolation order n_I, precision; owns the LGF table and kernel spectra."""

    def __init__(self, N: int = 16, n_interp: int = 6, precision: str = "fp64", max_oct_levels: int = 6,
                 table_radius: int = 100, asym_radius: int = 600, device: int | None = None):
        if not torch.cuda.is_available():
            raise FLGFError("the FLGF library needs a CUDA GPU; there is no CPU path")
        self.lib = load_library()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.N = int(N)
        self.n_interp = int(n_interp)
        self.precision = precision.lower()
        if self.precision not in ("fp64", "fp32"):
            raise ValueError("precision must be 'fp64' or 'fp32'")
        self.dtype = torch.float64 if self.precision == "fp64" else torch.float32
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.Stream(device=self.device)
        o = _Opts()
        self.lib.flgf_default_opts(ctypes.byref(o))
        o.N, o.n_interp = self.N, self.n_interp
        o.precision = FLGF_FP64 if self.precision == "fp64" else FLGF_FP32
        o.max_oct_levels, o.table_radius, o.asym_radius = max_oct_levels, table_radius, asym_radius
        o.stream = ctypes.c_void_p(self.stream.cuda_stream)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.lib.flgf_create(ctypes.byref(h), ctypes.byref(o))
        if rc != 0:
            raise FLGFError(f"flgf_create failed with code {rc}", rc)
        self.handle = h
        self.plan = (30, (4, 4, 8))  # (pair-list percentage, dense tile): the library's defaults

    def check(self, rc: int, what: str):
        if rc != 0:
            msg = self.lib.flgf_last_error(self.handle).decode()
            raise FLGFError(f"{what} failed ({rc}): {msg}", rc)

    def fail_alloc(self, n: int):
        """Failure injection: the n-th device allocation of this context's block
        sets from now on reports out-of-memory (0 disarms)."""
        self.check(self.lib.flgf_ctx_set_option(self.handle, CTX_FAIL_ALLOC, int(n)), "flgf_ctx_set_option")

    def set_plan(self, list_pct: int | None = None, tile=None):
        """Plan options for block sets created afterwards: the useful-pair
        percentage below which a tile runs on the pair-list MAC, and the dense
        MAC tile (t0, t1, t2) in parents."""
        if list_pct is not None:
            self.check(self.lib.flgf_ctx_set_option(self.handle, CTX_LIST_PCT, int(list_pct)), "flgf_ctx_set_option")
            self.plan = (int(list_pct), self.plan[1])
        if tile is not None:
            t = [int(v) for v in tile]
            self.check(self.lib.flgf_ctx_set_option(self.handle, CTX_TILE, t[0] | t[1] << 8 | t[2] << 16),
                       "flgf_ctx_set_option")
            self.plan = (self.plan[0], tuple(t))

    def lgf(self, pts) -> np.ndarray:
        pts = np.ascontiguousarray(np.asarray(pts, dtype=np.int32).reshape(-1, 3))
        out = np.empty(pts.shape[0], dtype=np.float64)
        self.check(self.lib.flgf_lgf_eval(self.handle, pts.shape[0], _ptr(pts, ctypes.c_int32),
                                          _ptr(out, ctypes.c_double)), "flgf_lgf_eval")
        return out

    def kernel_spectrum(self, k: int, d) -> np.ndarray:
        N = self.N
        out = np.empty(2 * (2 * N) * (2 * N) * (N + 1), dtype=np.float64)
        self.check(self.lib.flgf_kernel_spectrum(self.handle, k, int(d[0]), int(d[1]), int(d[2]),
                                                 _ptr(out, ctypes.c_double)), "flgf_kernel_spectrum")
        return out.view(np.complex128).reshape(2 * N, 2 * N, N + 1)

    def convolve_static(self, coords, f: torch.Tensor, h: float = 1.0, out: torch.Tensor | None = None):
        """Exact block convolution of at most 32 blocks (one 4x4x4 aligned box) with
        no device allocation inside the library; f and out are device tensors."""
        coords = np.ascontiguousarray(np.asarray(coords, dtype=np.int32).reshape(-1, 3))
        shape = (coords.shape[0], self.N, self.N, self.N)
        if not isinstance(f, torch.Tensor) or tuple(f.shape) != shape:
            raise ValueError(f"f must be a tensor of shape {shape}")
        f = f.to(device=self.device, dtype=self.dtype).contiguous()
        if out is None:
            out = torch.empty_like(f)
        elif (tuple(out.shape) != shape or out.dtype != self.dtype or out.device != self.device
              or not out.is_contiguous()):
            raise ValueError(f"out must be a contiguous {self.dtype} tensor of shape {shape} on {self.device}")
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self.check(self.lib.flgf_convolve_static(self.handle, coords.shape[0], _ptr(coords, ctypes.c_int32),
                                                 ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                                 float(h)), "flgf_convolve_static")
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        f.record_stream(self.stream)
        return out

    def refine_level(self, f: torch.Tensor, coords, rel: float):
        """One refinement step on the device (flgf_refine_level, Eq. ref_crit):
        f (nblk, N, N, N) the level's source, coords (nblk, 3) its block
        coordinates, rel = alpha^(L_R - l).  Returns device tensors (flags (nblk,)
        bool, children (m, 3) int32, buffer (k, 3) int32), the lists in Morton order."""
        coords = torch.as_tensor(coords, dtype=torch.int32).reshape(-1, 3).to(self.device).contiguous()
        n = coords.shape[0]
        shape = (n, self.N, self.N, self.N)
        if not isinstance(f, torch.Tensor) or tuple(f.shape) != shape:
            raise ValueError(f"f must be a tensor of shape {shape}")
        f = f.to(device=self.device, dtype=self.dtype).contiguous()
        flags = torch.empty(n, dtype=torch.uint8, device=self.device)
        children = torch.empty((8 * n, 3), dtype=torch.int32, device=self.device)
        buffer = torch.empty((26 * n, 3), dtype=torch.int32, device=self.device)
        counts = (ctypes.c_int * 2)()
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self.check(self.lib.flgf_refine_level(self.handle, ctypes.c_void_p(f.data_ptr()), n,
                                              ctypes.c_void_p(coords.data_ptr()), float(rel),
                                              ctypes.c_void_p(flags.data_ptr()), ctypes.c_void_p(children.data_ptr()),
                                              ctypes.c_void_p(buffer.data_ptr()), counts), "flgf_refine_level")
        return flags.bool(), children[:counts[0]], buffer[:counts[1]]

    def close(self):
        if getattr(self, "handle", None):
            self.lib.flgf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BlockSet:
    """One or more independent (possibly refined) Poisson problems.

    problems: list over problems of lists over levels of int (nb, 3) block
    coordinates; h0: per-problem spacing of level 0; want (optional): the same
    nesting of boolean arrays (nb,) marking the blocks whose potential is
    needed (a shard of a multi-GPU solve); the others are left unspecified.
    """

    def __init__(self, ctx: Context, problems, h0, want=None, vector: bool = False):
        """vector: the problems are the components of one vector field on one
        mesh (flgf_blockset_create_vector): every entry of problems must be the
        same mesh and every h0 the same spacing."""
        self.ctx = ctx
        self.lib = ctx.lib
        self.levels = [[np.asarray(c, dtype=np.int32).reshape(-1, 3) for c in p] for p in problems]
        nlev = np.array([len(p) for p in self.levels], dtype=np.int32)
        nblk = np.array([c.shape[0] for p in self.levels for c in p], dtype=np.int32)
        coords = np.ascontiguousarray(np.concatenate([c for p in self.levels for c in p], axis=0).astype(np.int32))
        h0 = np.ascontiguousarray(np.asarray(h0, dtype=np.float64).reshape(-1))
        if h0.size != len(self.levels):
            raise ValueError("one h0 per problem")
        h = ctypes.c_void_p()
        with torch.cuda.device(ctx.device):
            if vector:
                first = self.levels[0]
                if want is not None or np.any(h0 != h0[0]) or any(
                        len(p) != len(first) or any(not np.array_equal(a, b) for a, b in zip(p, first))
                        for p in self.levels):
                    raise ValueError("a vector block set takes one mesh, one h0 and no target mask")
                c0 = np.ascontiguousarray(np.concatenate(first, axis=0).astype(np.int32))
                nb0 = np.array([c.shape[0] for c in first], dtype=np.int32)
                rc = self.lib.flgf_blockset_create_vector(ctx.handle, len(self.levels), len(first),
                                                          _ptr(nb0, ctypes.c_int), _ptr(c0, ctypes.c_int32),
                                                          float(h0[0]), ctypes.byref(h))
            elif want is None:
                rc = self.lib.flgf_blockset_create(ctx.handle, len(self.levels), _ptr(nlev, ctypes.c_int),
                                                   _ptr(nblk, ctypes.c_int), _ptr(coords, ctypes.c_int32),
                                                   _ptr(h0, ctypes.c_double), ctypes.byref(h))
            else:
                w = np.ascontiguousarray(np.concatenate([np.asarray(m, dtype=bool).reshape(-1) for p in want for m in p])
                                         .astype(np.uint8))
                if w.size != coords.shape[0]:
                    raise ValueError("want must hold one flag per block")
                rc = self.lib.flgf_blockset_create_masked(ctx.handle, len(self.levels), _ptr(nlev, ctypes.c_int),
                                                          _ptr(nblk, ctypes.c_int), _ptr(coords, ctypes.c_int32),
                                                          _ptr(h0, ctypes.c_double), _ptr(w, ctypes.c_uint8),
                                                          ctypes.byref(h))
        ctx.check(rc, "flgf_blockset_create")
        self.handle = h
        self.h0 = h0

    @property
    def dof(self) -> int:
        return int(self.lib.flgf_blockset_dof(self.handle))

    def work_counts(self):
        v = [ctypes.c_int64() for _ in range(4)]
        self.ctx.check(self.lib.flgf_work_counts(self.handle, *[ctypes.byref(x) for x in v]), "flgf_work_counts")
        return dict(zip(("pairs", "fwd_ffts", "inv_ffts", "kernel_offsets"), (x.value for x in v)))

    def launch_count(self) -> int:
        """Kernels enqueued by the last solve."""
        return int(self.lib.flgf_launch_count(self.handle))

    def nblk(self, problem: int, level: int) -> int:
        return self.levels[problem][level].shape[0]

    def _shape(self, problem, level):
        N = self.ctx.N
        return (self.nblk(problem, level), N, N, N)

    def load_source(self, problem: int, level: int, f):
        """f: tensor or array of shape (nblk, N, N, N); converted to the context dtype."""
        shape = self._shape(problem, level)
        t = torch.as_tensor(f)
        if tuple(t.shape) != shape:
            raise ValueError(f"source shape {tuple(t.shape)} != {shape}")
        if t.is_cuda:
            t = t.to(dtype=self.ctx.dtype).contiguous()
            self.ctx.stream.wait_stream(torch.cuda.current_stream(t.device))
            where = FLGF_DEVICE
            keep = t
        else:
            keep = t.to(dtype=self.ctx.dtype).contiguous().numpy()
            where = FLGF_HOST
        ptr = keep.data_ptr() if where == FLGF_DEVICE else keep.ctypes.data
        self.ctx.check(self.lib.flgf_load_source(self.handle, problem, level, ctypes.c_void_p(ptr), where),
                       "flgf_load_source")
        if where == FLGF_DEVICE:
            keep.record_stream(self.ctx.stream)

    def solve(self):
        self.ctx.check(self.lib.flgf_solve(self.handle), "flgf_solve")

    def potential(self, problem: int = 0, level: int = 0, out: torch.Tensor | None = None) -> torch.Tensor:
        """u on the level's blocks, as a device tensor (nblk, N, N, N)."""
        shape = self._shape(problem, level)
        if out is None:
            out = torch.empty(shape, dtype=self.ctx.dtype, device=self.ctx.device)
        self.ctx.stream.wait_stream(torch.cuda.current_stream(self.ctx.device))
        self.ctx.check(self.lib.flgf_get_potential(self.handle, problem, level, ctypes.c_void_p(out.data_ptr()),
                                                   FLGF_DEVICE), "flgf_get_potential")
        torch.cuda.current_stream(self.ctx.device).wait_stream(self.ctx.stream)
        return out

    def load_adjoint(self, problem: int, level: int, g):
        """Adjoint seed dL/du of (problem, level), shape (nblk, N, N, N)."""
        shape = self._shape(problem, level)
        t = torch.as_tensor(g).to(device=self.ctx.device, dtype=self.ctx.dtype).contiguous()
        if tuple(t.shape) != shape:
            raise ValueError(f"adjoint shape {tuple(t.shape)} != {shape}")
        self.ctx.stream.wait_stream(torch.cuda.current_stream(self.ctx.device))
        self.ctx.check(self.lib.flgf_load_adjoint(self.handle, problem, level, ctypes.c_void_p(t.data_ptr()),
                                                  FLGF_DEVICE), "flgf_load_adjoint")
        t.record_stream(self.ctx.stream)

    def solve_adjoint(self):
        self.ctx.check(self.lib.flgf_solve_adjoint(self.handle), "flgf_solve_adjoint")

    def gradient(self, problem: int = 0, level: int = 0) -> torch.Tensor:
        """dL/df of (problem, level) after solve_adjoint, as a device tensor."""
        out = torch.empty(self._shape(problem, level), dtype=self.ctx.dtype, device=self.ctx.device)
        self.ctx.stream.wait_stream(torch.cuda.current_stream(self.ctx.device))
        self.ctx.check(self.lib.flgf_get_gradient(self.handle, problem, level, ctypes.c_void_p(out.data_ptr()),
                                                  FLGF_DEVICE), "flgf_get_gradient")
        torch.cuda.current_stream(self.ctx.device).wait_stream(self.ctx.stream)
        return out

    def keys(self):
        return [(p, l) for p in range(len(self.levels)) for l in range(len(self.levels[p]))]

    def potential_host(self, problem: int = 0, level: int = 0, out: np.ndarray | None = None) -> np.ndarray:
        """u into host memory (``out``: e.g. a pinned buffer of the right shape and dtype)."""
        dt = np.float64 if self.ctx.precision == "fp64" else np.float32
        if out is None:
            out = np.empty(self._shape(problem, level), dtype=dt)
        if out.dtype != dt or tuple(out.shape) != self._shape(problem, level) or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous array of the level's shape and the context dtype")
        self.ctx.check(self.lib.flgf_get_potential(self.handle, problem, level, ctypes.c_void_p(out.ctypes.data),
                                                   FLGF_HOST), "flgf_get_potential")
        return out

    def laplacian(self, problem: int, level: int, u) -> torch.Tensor:
        shape = self._shape(problem, level)
        u = torch.as_tensor(u).to(device=self.ctx.device, dtype=self.ctx.dtype).contiguous()
        if tuple(u.shape) != shape:
            raise ValueError("u shape mismatch")
        out = torch.empty_like(u)
        self.ctx.stream.wait_stream(torch.cuda.current_stream(self.ctx.device))
        self.ctx.check(self.lib.flgf_laplacian(self.handle, problem, level, ctypes.c_void_p(u.data_ptr()),
                                               ctypes.c_void_p(out.data_ptr()), FLGF_DEVICE), "flgf_laplacian")
        torch.cuda.current_stream(self.ctx.device).wait_stream(self.ctx.stream)
        u.record_stream(self.ctx.stream)
        return out

    def set_option(self, key: int, value: int):
        self.ctx.check(self.lib.flgf_set_option(self.handle, key, int(value)), "flgf_set_option")

    def stage_times(self, reset: bool = False):
        ms = np.zeros(len(STAGES))
        n = ctypes.c_int()
        self.ctx.check(self.lib.flgf_stage_times(self.handle, _ptr(ms, ctypes.c_double), len(STAGES), ctypes.byref(n),
                                                 int(reset)), "flgf_stage_times")
        return dict(zip(STAGES, ms.tolist())), n.value

    def close(self):
        if getattr(self, "handle", None):
            self.lib.flgf_blockset_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_problem(ctx: Context, prob, correction: bool = True, compensated: bool | None = None) -> list:
    """Convenience: solve one inputs.Problem; returns u per level as device tensors.
    compensated: FLGF_OPT_COMPENSATED (None keeps the library's default)."""
    bs = BlockSet(ctx, [prob.coords], [prob.h0])
    if not correction:
        bs.set_option(OPT_CORRECTION, 0)
    if compensated is not None:
        bs.set_option(OPT_COMPENSATED, int(compensated))
    for l, f in enumerate(prob.f):
        bs.load_source(0, l, torch.as_tensor(np.asarray(f)))
    bs.solve()
    out = [bs.potential(0, l) for l in range(len(prob.f))]
    torch.cuda.synchronize(ctx.device)
    bs.close()
    return out


def solve_vector(ctx: Context, coords_levels, h0: float, components, correction: bool = True) -> list:
    """Vector Poisson problem (each Cartesian component of a field, e.g. the
    streamfunction of a vorticity field, is a scalar problem on the same mesh):
    all components run as problems of one vector block set, so every stage of
    every component shares the same kernel launches and the same cached kernel
    spectra, and the spectrum products of three FP32 components share their
    kernel-spectrum reads.  components[c][l] is component c's source on level l; returns the
    potentials as components[c][l] device tensors."""
    bs = BlockSet(ctx, [coords_levels] * len(components), [h0] * len(components), vector=True)
    try:
        if not correction:
            bs.set_option(OPT_CORRECTION, 0)
        for c, levels in enumerate(components):
            for l, f in enumerate(levels):
                bs.load_source(c, l, torch.as_tensor(f))
        bs.solve()
        out = [[bs.potential(c, l) for l in range(len(coords_levels))] for c in range(len(components))]
        torch.cuda.synchronize(ctx.device)
        return out
    finally:
        bs.close()
