"""GB300 tensor butterfly: Python binding of the C ABI in include/tb.h.

Argument marshalling only: every step of construction and apply runs in the
CUDA library libtb.so (built by paper_2411_03029_gb300.build).  There is no CPU
fallback; a missing library raises.

  op = TBOperator(kind, d, n, xs, ys, tol, params=...)   # tb_build_ex (Alg. 1)
  u = op.apply(f)                                        # tb_apply   (Alg. 2), torch CUDA tensor
  v = op.apply_adjoint(g)                                # tb_apply_adjoint (K^H)
  u = apply(op, f)                                       # autograd: backward = adjoint apply
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

TB_MAX_D = 6
TB_MAX_LEVELS = 16

KERNEL_FOURIER, KERNEL_HELMHOLTZ, KERNEL_RADON, KERNEL_RADON_ANISO = 1, 2, 3, 4
PREC_C128, PREC_C64, PREC_C64_SPLITBF16 = 0, 1, 2
SEP_RULE, SEP_FIBER, SEP_TILE, SEP_REGISTER, SEP_REGISTER_PAIRS, SEP_REGISTER_SCALAR, SEP_REGISTER_ONE = range(7)
LEVEL_RULE, LEVEL_PER_MODE, LEVEL_FUSED, LEVEL_TENSOR = range(4)
CORE_RULE, CORE_STORED, CORE_REGENERATE = range(3)
ORDER_AUTO, ORDER_NATURAL, ORDER_BITREV = -1, 0, 1

STATUS = {0: "TB_OK", 1: "TB_EINVAL", 2: "TB_ENOMEM", 3: "TB_ECUDA", 4: "TB_ERANK",
          5: "TB_ETIMEOUT", 6: "TB_EUNSUPPORTED"}

# every symbol declared in include/tb.h
EXPORTS = ("tb_options_default", "tb_build", "tb_build_ex", "tb_apply", "tb_apply_adjoint",
           "tb_apply_host", "tb_query", "tb_free", "tb_last_error", "tb_version",
           "tb_profile_enable", "tb_profile_stats", "tb_apply_noalloc", "tb_autotune", "tb_apply_host_batch",
           "tb_alu_peak", "tb_cgls",
           "tb_export_factors", "tb_export_cores", "tb_export_order",
           "tb_apply_src_part", "tb_apply_tgt_part", "tb_shard_plan")


class TBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Kernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("params", ctypes.c_double * 4)]


class _Grids(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p * TB_MAX_D), ("y", ctypes.c_void_p * TB_MAX_D)]


class _Options(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("order", ctypes.c_int), ("proxy_rows", ctypes.c_int),
                ("rank_max", ctypes.c_int), ("precisions", ctypes.c_uint), ("separable", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("device", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("autotune", ctypes.c_int), ("sep_schedule", ctypes.c_int), ("level_schedule", ctypes.c_int),
                ("core_mode", ctypes.c_int), ("mode_slices", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("L", ctypes.c_int), ("Lc", ctypes.c_int), ("order", ctypes.c_int),
                ("separable", ctypes.c_int), ("n", ctypes.c_int64 * TB_MAX_D), ("cb", ctypes.c_int64 * TB_MAX_D),
                ("rank_src", (ctypes.c_int * TB_MAX_D) * TB_MAX_LEVELS),
                ("rank_tgt", (ctypes.c_int * TB_MAX_D) * TB_MAX_LEVELS),
                ("rank_min", ctypes.c_int), ("rank_max", ctypes.c_int), ("num_ids", ctypes.c_int64),
                ("core_entries", ctypes.c_int64), ("factor_entries", ctypes.c_int64),
                ("level_entries_max", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("build_seconds", ctypes.c_double), ("mid_src_entries", ctypes.c_int64),
                ("mid_tgt_entries", ctypes.c_int64)]


class _PassStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("level", ctypes.c_int), ("adjoint", ctypes.c_int),
                ("launches", ctypes.c_int64), ("ms_total", ctypes.c_double), ("bytes", ctypes.c_int64),
                ("flops", ctypes.c_double), ("kernels", ctypes.c_int64)]


_LIB = None


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libtb.so.  Raises if it has not been built: there is no fallback."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; build it with "
                               "paper_2411_03029_gb300.build.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(path)
        P, I64 = ctypes.c_void_p, ctypes.c_int64
        L.tb_options_default.argtypes = [ctypes.POINTER(_Options)]
        L.tb_build.argtypes = [ctypes.POINTER(_Kernel), ctypes.c_int, P, ctypes.POINTER(_Grids), ctypes.c_double,
                               ctypes.POINTER(P)]
        L.tb_build_ex.argtypes = [ctypes.POINTER(_Kernel), ctypes.c_int, P, ctypes.POINTER(_Grids), ctypes.c_double,
                                  ctypes.POINTER(_Options), ctypes.POINTER(P)]
        L.tb_apply.argtypes = [P, P, P, I64, ctypes.c_int, P]
        L.tb_apply_adjoint.argtypes = [P, P, P, I64, ctypes.c_int, P]
        L.tb_apply_host.argtypes = [P, P, P, I64, ctypes.c_int]
        L.tb_query.argtypes = [P, ctypes.POINTER(_Info)]
        L.tb_free.argtypes = [P]
        L.tb_last_error.argtypes = []
        L.tb_last_error.restype = ctypes.c_char_p
        L.tb_version.argtypes = []
        L.tb_version.restype = ctypes.c_char_p
        L.tb_profile_enable.argtypes = [P, ctypes.c_int]
        L.tb_profile_stats.argtypes = [P, ctypes.POINTER(_PassStat), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.tb_apply_noalloc.argtypes = [P, P, P, I64, ctypes.c_int, P]
        L.tb_apply_host_batch.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), I64, I64, ctypes.c_int]
        L.tb_alu_peak.argtypes = [ctypes.c_int, P, ctypes.POINTER(ctypes.c_double)]
        L.tb_cgls.argtypes = [P, P, P, I64, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]
        L.tb_export_factors.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P]
        L.tb_export_cores.argtypes = [P, P, P, P, P, P]
        L.tb_export_order.argtypes = [P, ctypes.c_int, P]
        L.tb_apply_src_part.argtypes = [P, P, P, I64, I64, I64, ctypes.c_int, P]
        L.tb_apply_tgt_part.argtypes = [P, P, P, I64, I64, I64, ctypes.c_int, P]
        L.tb_shard_plan.argtypes = [I64, ctypes.c_int, P, P]
        for name in ("tb_options_default", "tb_build", "tb_build_ex", "tb_apply", "tb_apply_adjoint",
                     "tb_apply_host", "tb_query", "tb_free", "tb_profile_enable", "tb_profile_stats",
                     "tb_apply_noalloc", "tb_apply_host_batch", "tb_alu_peak", "tb_cgls",
                     "tb_export_factors", "tb_export_cores", "tb_export_order",
                     "tb_apply_src_part", "tb_apply_tgt_part", "tb_shard_plan"):
            getattr(L, name).restype = ctypes.c_int
        _LIB = L
    return _LIB


def _check(status: int):
    if status != 0:
        raise TBError(status, lib().tb_last_error().decode())


def _torch():
    import torch
    return torch


def dtype_of(precision: int):
    torch = _torch()
    return torch.complex128 if precision == PREC_C128 else torch.complex64


class TBOperator:
    """A tensor butterfly of K on tensor grids, built on the current CUDA device."""

    def __init__(self, kind: int, d: int, n, xs, ys, tol: float, params=(), L: int = -1,
                 order: int = ORDER_AUTO, precisions: int = 0, separable: int = -1,
                 use_graphs: bool = False, proxy_rows: int = 1024, rank_max: int = 32,
                 seed: int = 0x5eed, precision: int = PREC_C64, autotune: bool = False,
                 sep_schedule: int = 0, level_schedule: int = 0, core_mode: int = 0, mode_slices: int = 0):
        L_ = lib()
        n = [int(v) for v in (n if np.iterable(n) else [n] * d)]
        self.d, self.n, self.kind = d, n, kind
        self.precision = precision
        self._xs = [np.ascontiguousarray(x, dtype=np.float64) for x in xs]
        self._ys = [np.ascontiguousarray(y, dtype=np.float64) for y in ys]
        kern = _Kernel(kind, (ctypes.c_double * 4)(*(list(params) + [0.0] * (4 - len(params)))))
        grids = _Grids()
        for k in range(d):
            grids.x[k] = self._xs[k].ctypes.data
            grids.y[k] = self._ys[k].ctypes.data
        opt = _Options()
        _check(L_.tb_options_default(ctypes.byref(opt)))
        opt.L, opt.order, opt.proxy_rows, opt.rank_max = L, order, proxy_rows, rank_max
        opt.precisions, opt.separable, opt.use_graphs, opt.seed = precisions, separable, int(use_graphs), seed
        opt.autotune = int(autotune)
        opt.sep_schedule = int(sep_schedule)
        opt.level_schedule = int(level_schedule)
        opt.core_mode = int(core_mode)
        opt.mode_slices = int(mode_slices)
        try:
            opt.device = _torch().cuda.current_device()
        except Exception:  # pragma: no cover
            opt.device = -1
        narr = (ctypes.c_int64 * d)(*n)
        h = ctypes.c_void_p()
        _check(L_.tb_build_ex(ctypes.byref(kern), d, ctypes.cast(narr, ctypes.c_void_p), ctypes.byref(grids),
                              float(tol), ctypes.byref(opt), ctypes.byref(h)))
        self._h = h

    @property
    def N(self) -> int:
        return int(np.prod(self.n))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().tb_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        inf = _Info()
        _check(lib().tb_query(self._h, ctypes.byref(inf)))
        Lc = inf.Lc
        return {
            "d": inf.d, "L": inf.L, "Lc": Lc, "order": inf.order, "separable": inf.separable,
            "n": list(inf.n[: inf.d]), "cb": list(inf.cb[: inf.d]),
            "rank_src": [list(inf.rank_src[l][: inf.d]) for l in range(Lc + 1)],
            "rank_tgt": [list(inf.rank_tgt[l][: inf.d]) for l in range(Lc + 1)],
            "rank_min": inf.rank_min, "rank_max": inf.rank_max, "num_ids": inf.num_ids,
            "core_entries": inf.core_entries, "factor_entries": inf.factor_entries,
            "level_entries_max": inf.level_entries_max, "device_bytes": inf.device_bytes,
            "build_seconds": inf.build_seconds,
            "mid_src_entries": inf.mid_src_entries, "mid_tgt_entries": inf.mid_tgt_entries,
        }

    def autotune(self, nv: int = 1, precision: int | None = None):
        """Tune the launch shapes for nv RHS at `precision` on the current stream (tb_autotune)."""
        torch = _torch()
        precision = self.precision if precision is None else precision
        _check(lib().tb_autotune(self._h, int(nv), precision,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))

    def profile(self, on: bool = True):
        """Record CUDA events around every pass of eager applies (tb_profile_enable)."""
        _check(lib().tb_profile_enable(self._h, int(on)))

    def profile_stats(self) -> list:
        """Per-pass launches, device time, bytes and flops since the last call."""
        arr = (_PassStat * 64)()
        cnt = ctypes.c_int()
        _check(lib().tb_profile_stats(self._h, arr, 64, ctypes.byref(cnt)))
        return [{"name": a.name.decode(), "level": a.level, "adjoint": a.adjoint, "launches": a.launches,
                 "ms_total": a.ms_total, "bytes": a.bytes, "flops": a.flops, "kernels": a.kernels}
                for a in arr[: cnt.value]]

    def _prep(self, x, precision):
        torch = _torch()
        precision = self.precision if precision is None else precision
        dt = dtype_of(precision)
        if not isinstance(x, torch.Tensor) or not x.is_cuda:
            raise TypeError("expected a CUDA torch tensor")
        if x.dtype != dt:
            raise TypeError(f"precision {precision} needs dtype {dt}, got {x.dtype}")
        squeeze = x.dim() == self.d
        if squeeze:
            x = x.unsqueeze(-1)
        if tuple(x.shape[: self.d]) != tuple(self.n) or x.dim() != self.d + 1:
            raise ValueError(f"expected shape {tuple(self.n)} + (nv,), got {tuple(x.shape)}")
        if not x.is_contiguous():
            x = x.contiguous()
        return x, precision, squeeze

    def _run(self, fn, x, precision, out):
        torch = _torch()
        x, precision, squeeze = self._prep(x, precision)
        nv = x.shape[-1]
        if out is None:
            out = torch.empty_like(x)
        stream = torch.cuda.current_stream(x.device).cuda_stream
        _check(fn(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), nv, precision,
                  ctypes.c_void_p(stream)))
        return out.squeeze(-1) if squeeze else out

    def apply(self, f, precision: int | None = None, out=None):
        """u = K f on the current torch stream (tb_apply)."""
        return self._run(lib().tb_apply, f, precision, out)

    def apply_adjoint(self, g, precision: int | None = None, out=None):
        """v = K^H g on the current torch stream (tb_apply_adjoint)."""
        return self._run(lib().tb_apply_adjoint, g, precision, out)

    def cgls(self, b, iters: int, x0=None, precision: int | None = None, graph: bool = True):
        """Least squares min_x ||K x - b|| per RHS column by CGLS on the device (tb_cgls).

        b: CUDA tensor of the target-grid shape (+ nv); x0: start (zeros if None).
        Returns (x, resid) with resid[k, v] = ||b - K x_k|| of column v after k
        iterations (numpy, (iters + 1) x nv).  With graph=True one iteration is
        captured as a CUDA graph and replayed on the current stream."""
        torch = _torch()
        b, precision, squeeze = self._prep(b, precision)
        nv = b.shape[-1]
        x = torch.zeros_like(b) if x0 is None else self._prep(x0, precision)[0].clone()
        resid = np.zeros((iters + 1, nv), dtype=np.float64)
        stream = torch.cuda.current_stream(b.device).cuda_stream
        _check(lib().tb_cgls(self._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), nv,
                             int(iters), precision, int(graph), ctypes.c_void_p(resid.ctypes.data),
                             ctypes.c_void_p(stream)))
        return (x.squeeze(-1) if squeeze else x), resid

    def export(self) -> dict:
        """The built butterfly as host arrays (tb_export_factors / _cores / _order):
        {"d", "L", "Lc", "n", "cb", "perm": [d int arrays],
         "factors": {(side, level, mode): {"ranks", "skel", "blocks"}},
         "core_offsets", "core_dims", "core"}.  See include/tb.h for the indexing."""
        L_ = lib()
        inf = self.info()
        d, Lc = inf["d"], inf["Lc"]
        out = {"d": d, "L": inf["L"], "Lc": Lc, "n": inf["n"], "cb": inf["cb"], "perm": [], "factors": {}}
        for k in range(d):
            perm = np.zeros(inf["n"][k], dtype=np.int32)
            _check(L_.tb_export_order(self._h, k, ctypes.c_void_p(perm.ctypes.data)))
            out["perm"].append(perm)
        cnt, rows, cols = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        for side in (0, 1):
            for lvl in range(Lc + 1):
                for k in range(d):
                    _check(L_.tb_export_factors(self._h, side, lvl, k, ctypes.byref(cnt), ctypes.byref(rows),
                                                ctypes.byref(cols), None, None, None))
                    ranks = np.zeros(cnt.value, dtype=np.int32)
                    skel = np.zeros((cnt.value, rows.value), dtype=np.int32)
                    blocks = np.zeros((cnt.value, rows.value, cols.value), dtype=np.complex128)
                    _check(L_.tb_export_factors(self._h, side, lvl, k, ctypes.byref(cnt), ctypes.byref(rows),
                                                ctypes.byref(cols), ctypes.c_void_p(ranks.ctypes.data),
                                                ctypes.c_void_p(skel.ctypes.data),
                                                ctypes.c_void_p(blocks.ctypes.data)))
                    out["factors"][(side, lvl, k)] = {"ranks": ranks, "skel": skel, "blocks": blocks}
        pairs, entries = ctypes.c_int64(), ctypes.c_int64()
        _check(L_.tb_export_cores(self._h, ctypes.byref(pairs), ctypes.byref(entries), None, None, None))
        offs = np.zeros(pairs.value + 1, dtype=np.int64)
        dims = np.zeros((pairs.value, 2 * d), dtype=np.int32)
        core = np.zeros(entries.value, dtype=np.complex128)
        _check(L_.tb_export_cores(self._h, ctypes.byref(pairs), ctypes.byref(entries), ctypes.c_void_p(offs.ctypes.data),
                                  ctypes.c_void_p(dims.ctypes.data), ctypes.c_void_p(core.ctypes.data)))
        out.update(core_offsets=offs, core_dims=dims, core=core)
        return out

    # ------------------------------------------------------ partitioned apply
    def mid_shape(self, nv: int) -> tuple:
        """Shape (nF, nF, tile entries, nv) of the mid-level tensor exchanged by a
        partitioned apply (tb_apply_src_part / tb_apply_tgt_part)."""
        inf = self.info()
        nF = 2 ** (inf["d"] * inf["Lc"])
        return (nF, nF, int(np.prod(inf["rank_tgt"][inf["Lc"]])), int(nv))

    def apply_src_part(self, f, g_mid, s_range, precision: int | None = None):
        """Steps 1 and 2 of Alg. 2 for the mid-level source multi-sets in s_range = (begin, end):
        writes the mid-level tiles (t, s) of those s into g_mid (tb_apply_src_part)."""
        torch = _torch()
        f, precision, _ = self._prep(f, precision)
        stream = torch.cuda.current_stream(f.device).cuda_stream
        _check(lib().tb_apply_src_part(self._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(g_mid.data_ptr()),
                                       f.shape[-1], int(s_range[0]), int(s_range[1]), precision,
                                       ctypes.c_void_p(stream)))
        return g_mid

    def apply_tgt_part(self, g_mid, u, t_range, precision: int | None = None):
        """Step 3 of Alg. 2 for the mid-level target multi-sets in t_range: writes the target
        points of those t into u (tb_apply_tgt_part)."""
        torch = _torch()
        u_, precision, _ = self._prep(u, precision)
        if u_.data_ptr() != u.data_ptr():
            raise ValueError("u must be a contiguous tensor of the apply layout")
        stream = torch.cuda.current_stream(u.device).cuda_stream
        _check(lib().tb_apply_tgt_part(self._h, ctypes.c_void_p(g_mid.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                       u_.shape[-1], int(t_range[0]), int(t_range[1]), precision,
                                       ctypes.c_void_p(stream)))
        return u

    def apply_host_batch(self, fs, us, precision: int | None = None):
        """u_i = K f_i for lists of host arrays (numpy, pinned for overlap), with the
        copies of neighbouring inputs and results overlapping the applies
        (tb_apply_host_batch).  Results are written into `us`."""
        precision = self.precision if precision is None else precision
        dt = np.complex128 if precision == PREC_C128 else np.complex64
        if len(fs) != len(us) or not fs:
            raise ValueError("fs and us must be non-empty lists of the same length")
        for a in list(fs) + list(us):
            if a.dtype != dt or not a.flags.c_contiguous:
                raise TypeError(f"host arrays must be C-contiguous {dt}")
        nv = fs[0].shape[-1] if fs[0].ndim == self.d + 1 else 1
        fp = (ctypes.c_void_p * len(fs))(*[a.ctypes.data for a in fs])
        up = (ctypes.c_void_p * len(us))(*[a.ctypes.data for a in us])
        _check(lib().tb_apply_host_batch(self._h, fp, up, len(fs), nv, precision))
        return us

    def apply_host(self, f: np.ndarray, precision: int | None = None) -> np.ndarray:
        """u = K f with host arrays; copies in and out inside the call (tb_apply_host)."""
        precision = self.precision if precision is None else precision
        dt = np.complex128 if precision == PREC_C128 else np.complex64
        f = np.ascontiguousarray(f, dtype=dt)
        nv = f.shape[-1] if f.ndim == self.d + 1 else 1
        u = np.empty_like(f)
        _check(lib().tb_apply_host(self._h, ctypes.c_void_p(f.ctypes.data), ctypes.c_void_p(u.ctypes.data),
                                   nv, precision))
        return u


def shard_plan(nmid: int, nranks: int):
    """Contiguous near-equal ranges [(begin, end)] of nmid mid-level multi-sets over nranks
    ranks (tb_shard_plan; host only)."""
    b = (ctypes.c_int64 * nranks)()
    e = (ctypes.c_int64 * nranks)()
    _check(lib().tb_shard_plan(int(nmid), int(nranks), b, e))
    return [(b[g], e[g]) for g in range(nranks)]


def sharded_apply(op, f, precision: int | None = None, group=None):
    """u = K f with the work partitioned over the ranks of a torch.distributed group,
    one operator (device) per rank (Sec. 3.2: steps 1 and 3 of Alg. 2 are independent per
    mid-level multi-set; the mid-level tiles are the one exchange):

      1. rank g runs steps 1-2 for its source range S_g (op.apply_src_part);
      2. the tiles (t, s), t in T_h, s in S_g, go to rank h: point-to-point
         sends and receives of contiguous blocks (all ranks at once);
      3. rank g runs step 3 for its target range T_g (op.apply_tgt_part).

    f must hold at least the source points of S_g.  Returns this rank's u: the
    target points of T_g are set, the others are zero (sum over the ranks for
    the whole result).  `op` needs apply_src_part, apply_tgt_part and
    mid_shape; tensors live on the device of f."""
    torch = _torch()
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    nv = f.shape[-1] if f.dim() == len(op.n) + 1 else 1
    shape = op.mid_shape(nv)
    nF = shape[0]
    plan = shard_plan(nF, world)
    dt = f.dtype
    g_mid = torch.zeros(shape, dtype=dt, device=f.device)
    s0, s1 = plan[rank]
    op.apply_src_part(f, g_mid, (s0, s1), precision)
    t0, t1 = plan[rank]
    reqs, recv = [], []
    for h in range(world):
        th0, th1 = plan[h]
        sh0, sh1 = plan[h]
        if h == rank:
            continue
        # complex tiles travel as their real views (re, im pairs)
        send = torch.view_as_real(g_mid[th0:th1, s0:s1].contiguous())
        buf = torch.empty((t1 - t0, sh1 - sh0) + tuple(shape[2:]), dtype=dt, device=f.device)
        peer = dist.get_global_rank(group, h) if group is not None else h
        if send.numel():
            reqs.append(dist.isend(send, dst=peer, group=group))
        if buf.numel():
            reqs.append(dist.irecv(torch.view_as_real(buf), src=peer, group=group))
        recv.append((sh0, sh1, buf, send))
    for r in reqs:
        r.wait()
    for sh0, sh1, buf, _ in recv:
        if buf.numel():
            g_mid[t0:t1, sh0:sh1] = buf
    u = torch.zeros_like(f)
    op.apply_tgt_part(g_mid, u, (t0, t1), precision)
    return u


def alu_peak(precision: int = PREC_C64) -> float:
    """Measured FMA throughput (TFLOP/s) of the current device: FP32 for PREC_C64,
    FP64 for PREC_C128 (tb_alu_peak)."""
    torch = _torch()
    out = ctypes.c_double()
    _check(lib().tb_alu_peak(int(precision), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                             ctypes.byref(out)))
    return out.value


def from_workload(w, **kw) -> TBOperator:
    """Build the operator of a workloads.Workload (grids, kernel, tolerance, order)."""
    import workloads
    xs, ys = workloads.grids(w)
    kw.setdefault("L", w.L)
    kw.setdefault("order", w.order)
    kw.setdefault("precision", w.precision)
    return TBOperator(w.kind, w.d, [w.n] * w.d, xs, ys, w.tol, params=w.params, **kw)


def _autograd_fn():
    torch = _torch()

    class TBApply(torch.autograd.Function):
        """u = K f with the adjoint butterfly as its backward.

        For a linear map, PyTorch's complex convention passes grad_u = dL/dRe(u)
        + i dL/dIm(u) and expects dL/dRe(f) + i dL/dIm(f) = K^H grad_u."""

        @staticmethod
        def forward(ctx, f, op, precision):
            ctx.op, ctx.precision = op, precision
            return op.apply(f.detach(), precision)

        @staticmethod
        def backward(ctx, gu):
            return ctx.op.apply_adjoint(gu.contiguous(), ctx.precision), None, None

    return TBApply


_TBApply = None


def apply(op: TBOperator, f, precision: int | None = None):
    """Differentiable u = K f (backward: v = K^H grad_u through tb_apply_adjoint)."""
    global _TBApply
    if _TBApply is None:
        _TBApply = _autograd_fn()
    return _TBApply.apply(f, op, op.precision if precision is None else precision)
