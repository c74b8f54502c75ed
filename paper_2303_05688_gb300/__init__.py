"""Python binding of libasci, the GB300 ASCI library (arXiv:2303.05688): the
determinant search (Alg. 2, Eq. 1) and its stages, batched and sharded
searches with a distributed top-N (the role of Alg. 4), the variational step
(Hamiltonian, sparse product, Davidson: Sec. 2.3, Alg. 5), the ASCI loop
(Alg. 1) and ASCI-PT2.

Argument marshalling only: every step runs in the CUDA kernels of
``lib/libasci.so`` behind the C ABI declared in ``include/asci.h``.  There is
no CPU fallback; importing works without a GPU, but every call needs the built
library and a CUDA device, and raises otherwise.

Arrays may be numpy arrays (host memory; the library copies them in) or torch
tensors on the CUDA device (used in place).  Determinants are uint64 pairs
(alpha word, beta word); torch tensors may hold them as int64 bit patterns.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass

import numpy as np

__all__ = ["load", "lib_path", "launch_count", "search", "excitations", "diagonal", "sort_accumulate",
           "select_topn", "SearchStats", "AsciError", "FP64", "FP32_INT_FP64_ACC",
           "FP32_INT_COMP_ACC", "shard_assign", "gather_candidates", "sharded_search",
           "search_many", "tune_streams", "tune_batched", "hamiltonian", "spmv", "davidson", "asci_loop",
           "LoopStats", "pt2", "select_histogram", "select_below", "distributed_topn",
           "constraint_classes"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "lib", "libasci.so")

FP64, FP32_INT_FP64_ACC, FP32_INT_COMP_ACC = 0, 1, 2
_ERRORS = {-1: "ASCI_EINVAL", -2: "ASCI_ENOMEM", -3: "ASCI_ECUDA", -4: "ASCI_ETIMEOUT"}


class AsciError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        super().__init__(f"{where}: {_ERRORS.get(code, code)}" + (f" ({detail})" if detail else ""))


class _Det(ct.Structure):
    _fields_ = [("alpha", ct.c_uint64), ("beta", ct.c_uint64)]


class _Ints(ct.Structure):
    _fields_ = [("norb", ct.c_int32), ("ecore", ct.c_double), ("h1", ct.c_void_p),
                ("eri", ct.c_void_p)]


class _Opts(ct.Structure):
    _fields_ = [("eps_search", ct.c_double), ("max_constraint_level", ct.c_int32),
                ("precision", ct.c_int32), ("max_batch_pairs", ct.c_uint64),
                ("sort_output", ct.c_int32), ("shard_index", ct.c_int32),
                ("shard_count", ct.c_int32), ("ctas_per_sm", ct.c_int32)]


class _SelectState(ct.Structure):
    _fields_ = [("prefix", ct.c_uint64 * 2), ("mask", ct.c_uint64 * 2),
                ("threshold", ct.c_uint64 * 2), ("remaining", ct.c_uint64),
                ("digit", ct.c_int32), ("done", ct.c_int32)]


class _Problem(ct.Structure):
    _fields_ = [("dets", ct.c_void_p), ("coeffs", ct.c_void_p), ("ndets", ct.c_size_t),
                ("E0", ct.c_double), ("ints", ct.c_void_p), ("C", ct.c_size_t),
                ("N", ct.c_size_t), ("out_dets", ct.c_void_p), ("out_scores", ct.c_void_p),
                ("out_n", ct.c_void_p), ("stats", ct.c_void_p), ("status", ct.c_int32)]


class _Stats(ct.Structure):
    _fields_ = [("generated", ct.c_uint64), ("surviving", ct.c_uint64), ("unique", ct.c_uint64),
                ("excluded", ct.c_uint64), ("selected", ct.c_uint64), ("batches", ct.c_uint64),
                ("max_batch", ct.c_uint64), ("ncore", ct.c_uint64), ("max_level", ct.c_uint64),
                ("tile_launches", ct.c_uint64), ("tile_records", ct.c_uint64),
                ("oversized_records", ct.c_uint64), ("diag_grid_bits", ct.c_uint64),
                ("big_tile_records", ct.c_uint64), ("t_stage", ct.c_double * 8)]


class _DavOpts(ct.Structure):
    _fields_ = [("max_subspace", ct.c_int32), ("max_iter", ct.c_int32), ("tol", ct.c_double)]


_MAX_STEPS = 64


class _LoopOpts(ct.Structure):
    _fields_ = [("ncdets", ct.c_uint64), ("ntdets", ct.c_uint64), ("max_steps", ct.c_int32),
                ("etol", ct.c_double), ("search", _Opts), ("davidson", _DavOpts)]


class _LoopStats(ct.Structure):
    _fields_ = [("steps", ct.c_int32), ("start_energy", ct.c_double),
                ("energy", ct.c_double * _MAX_STEPS), ("ndets", ct.c_uint64 * _MAX_STEPS),
                ("new_dets", ct.c_uint64 * _MAX_STEPS), ("nnz", ct.c_uint64 * _MAX_STEPS),
                ("davidson_iters", ct.c_int32 * _MAX_STEPS),
                ("t_search", ct.c_double * _MAX_STEPS),
                ("t_hamiltonian", ct.c_double * _MAX_STEPS),
                ("t_davidson", ct.c_double * _MAX_STEPS)]


@dataclass
class LoopStats:
    """Per-step record of asci_loop(): energies, sizes, H nonzeros, Davidson
    products and device milliseconds of the search, the build and Davidson."""
    start_energy: float
    energy: list
    ndets: list
    new_dets: list
    nnz: list
    davidson_iters: list
    t_search_ms: list
    t_hamiltonian_ms: list
    t_davidson_ms: list

    @classmethod
    def _from(cls, s: _LoopStats):
        k = s.steps
        return cls(s.start_energy, list(s.energy[:k]), list(s.ndets[:k]), list(s.new_dets[:k]),
                   list(s.nnz[:k]), list(s.davidson_iters[:k]), list(s.t_search[:k]),
                   list(s.t_hamiltonian[:k]), list(s.t_davidson[:k]))


@dataclass
class SearchStats:
    generated: int
    surviving: int
    unique: int
    excluded: int
    selected: int
    batches: int
    max_batch: int
    ncore: int
    max_level: int
    tile_launches: int
    tile_records: int
    oversized_records: int
    diag_grid_bits: int
    big_tile_records: int
    t_stage_ms: dict

    @classmethod
    def _from(cls, s: _Stats):
        names = ["prepare", "plan", "generate", "tiles", "oversized", "score", "select", "total"]
        return cls(s.generated, s.surviving, s.unique, s.excluded, s.selected, s.batches,
                   s.max_batch, s.ncore, s.max_level, s.tile_launches, s.tile_records,
                   s.oversized_records, s.diag_grid_bits, s.big_tile_records,
                   {k: s.t_stage[i] for i, k in enumerate(names)})


_lib = None


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libasci.so (built by paper_2303_05688_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"libasci.so is not built ({_LIB_PATH}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ct.CDLL(_LIB_PATH)
    vp, sz, szp = ct.c_void_p, ct.c_size_t, ct.POINTER(ct.c_size_t)
    lib.asci_search.restype = ct.c_int
    lib.asci_search.argtypes = [vp, vp, sz, ct.c_double, ct.POINTER(_Ints), sz, sz,
                                ct.POINTER(_Opts), vp, vp, szp, ct.POINTER(_Stats), vp]
    lib.asci_pt2.restype = ct.c_int
    lib.asci_pt2.argtypes = [vp, vp, sz, ct.c_double, ct.POINTER(_Ints), sz, ct.POINTER(_Opts),
                             ct.POINTER(ct.c_double), ct.POINTER(_Stats), vp]
    lib.asci_excitations.restype = ct.c_int
    lib.asci_excitations.argtypes = [ct.POINTER(_Ints), vp, vp, sz, vp, vp, sz, szp, vp]
    lib.asci_diagonal.restype = ct.c_int
    lib.asci_diagonal.argtypes = [ct.POINTER(_Ints), vp, sz, vp, vp]
    lib.asci_sort_accumulate.restype = ct.c_int
    lib.asci_sort_accumulate.argtypes = [vp, vp, sz, vp, vp, szp, vp]
    lib.asci_select_histogram.restype = ct.c_int
    lib.asci_select_histogram.argtypes = [vp, vp, sz, ct.c_int32, vp, vp, vp, vp]
    lib.asci_select_begin.restype = ct.c_int
    lib.asci_select_begin.argtypes = [ct.c_uint64, ct.c_uint64, ct.POINTER(_SelectState)]
    lib.asci_select_step.restype = ct.c_int
    lib.asci_select_step.argtypes = [ct.POINTER(_SelectState), vp]
    lib.asci_select_below.restype = ct.c_int
    lib.asci_select_below.argtypes = [vp, vp, sz, vp, vp, vp, szp, vp]
    lib.asci_select_topn.restype = ct.c_int
    lib.asci_select_topn.argtypes = [vp, vp, sz, sz, vp, vp, szp, vp]
    lib.asci_shard_assign.argtypes = [vp, sz, ct.c_int32, vp, vp]
    lib.asci_constraint_classes.restype = ct.c_int
    lib.asci_constraint_classes.argtypes = [vp, vp, sz, ct.POINTER(_Ints), sz, ct.c_int32, vp, sz,
                                            szp, vp]
    lib.asci_search_many.argtypes = [vp, sz, ct.POINTER(_Opts), ct.c_int32]
    lib.asci_default_opts.argtypes = [ct.POINTER(_Opts)]
    lib.asci_hamiltonian.restype = ct.c_int
    lib.asci_hamiltonian.argtypes = [vp, sz, ct.POINTER(_Ints), vp, vp, vp, sz, szp, vp]
    lib.asci_spmv.restype = ct.c_int
    lib.asci_spmv.argtypes = [vp, vp, vp, sz, vp, vp, vp]
    lib.asci_davidson.restype = ct.c_int
    lib.asci_davidson.argtypes = [vp, vp, vp, sz, vp, ct.POINTER(_DavOpts), vp, vp, vp, vp, vp]
    lib.asci_default_davidson_opts.argtypes = [ct.POINTER(_DavOpts)]
    lib.asci_default_loop_opts.argtypes = [ct.POINTER(_LoopOpts)]
    lib.asci_loop.restype = ct.c_int
    lib.asci_loop.argtypes = [vp, vp, sz, ct.POINTER(_Ints), ct.POINTER(_LoopOpts), vp, vp, sz,
                              szp, vp, ct.POINTER(_LoopStats), vp]
    lib.asci_version.restype = ct.c_char_p
    lib.asci_strerror.restype = ct.c_char_p
    lib.asci_strerror.argtypes = [ct.c_int]
    lib.asci_last_error.restype = ct.c_char_p
    lib.asci_launch_count.restype = ct.c_ulonglong
    lib.asci_trim_cache.restype = None
    lib.asci_debug_fail_allocation.restype = None
    lib.asci_debug_fail_allocation.argtypes = [ct.c_int64]
    _lib = lib
    return lib


def launch_count() -> int:
    """Kernels launched by libasci in this process so far."""
    return int(load().asci_launch_count())


def _check(code: int, where: str):
    if code != 0:
        detail = (load().asci_last_error() or b"").decode(errors="replace")
        raise AsciError(code, where, detail)


# ------------------------------- marshalling -------------------------------

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _torch():
    import torch
    return torch


class _Buf:
    """A contiguous buffer (host numpy or device torch) and its raw pointer."""

    def __init__(self, obj, ptr, device: bool):
        self.obj, self.ptr, self.device = obj, ptr, device


def _as_buf(x, np_dtype, torch_dtype_name):
    if _is_torch(x):
        torch = _torch()
        t = x.contiguous()
        want = getattr(torch, torch_dtype_name)
        if t.dtype != want:
            if torch_dtype_name == "int64" and t.dtype == getattr(torch, "uint64", None):
                t = t.view(torch.int64)
            else:
                t = t.to(want)
        if not t.is_cuda:
            t = t.cpu()
            return _Buf(t, t.data_ptr(), False)
        return _Buf(t, t.data_ptr(), True)
    a = np.ascontiguousarray(x, dtype=np_dtype)
    return _Buf(a, a.ctypes.data, False)


def _dets_buf(dets):
    """(n, 2) uint64 (alpha, beta) determinants, or a pair (alpha[n], beta[n])."""
    if isinstance(dets, tuple) and len(dets) == 2:
        a, b = dets
        if _is_torch(a):
            torch = _torch()
            d = torch.stack([a.view(torch.int64) if a.dtype != torch.int64 else a,
                             b.view(torch.int64) if b.dtype != torch.int64 else b], dim=1)
            return _as_buf(d, np.uint64, "int64")
        d = np.stack([np.asarray(a, dtype=np.uint64), np.asarray(b, dtype=np.uint64)], axis=1)
        return _as_buf(d, np.uint64, "int64")
    return _as_buf(dets, np.uint64, "int64")


def _stream_ptr(stream, device: bool):
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    if device:
        return int(_torch().cuda.current_stream().cuda_stream)
    return None


def _ints(h1, eri, ecore, keep):
    hb = _as_buf(h1, np.float64, "float64")
    eb = _as_buf(eri, np.float64, "float64")
    keep += [hb, eb]
    n = int(round(np.sqrt(np.prod(hb.obj.shape))))
    return _Ints(n, float(ecore), hb.ptr, eb.ptr), hb.device


def _out(n, dtype_np, device, cols=None):
    shape = (n, cols) if cols else (n,)
    if device:
        torch = _torch()
        tdt = {np.float64: torch.float64, np.uint64: torch.int64}[dtype_np]
        t = torch.empty(shape, dtype=tdt, device="cuda")
        return t, t.data_ptr()
    a = np.empty(shape, dtype=dtype_np)
    return a, a.ctypes.data


# --------------------------------- calls -----------------------------------

def search(dets, coeffs, E0: float, h1, eri, ecore: float, C: int, N: int, *,
           eps: float = 0.0, precision: int = FP64, max_batch_pairs: int = 0,
           max_constraint_level: int = 0, sort_output: bool = False, stream=None,
           return_stats: bool = True, shard=None, ctas_per_sm: int = 0):
    """The ASCI search (Alg. 2 with Eq. 1).  Returns (dets[(m, 2)], scores[m], stats).

    Outputs live where ``dets`` lives (device torch tensors in, device tensors out).
    ``shard=(index, count)`` restricts the search to one shard of the target
    alpha classes (Sec. 2.2, Alg. 3) and returns that shard's top N.
    ``ctas_per_sm`` caps the persistent kernels' CTAs per SM (0: as many as fit).
    """
    lib = load()
    keep = []
    db = _dets_buf(dets)
    cb = _as_buf(coeffs, np.float64, "float64")
    keep += [db, cb]
    ints, _ = _ints(h1, eri, ecore, keep)
    nd = int(db.obj.shape[0])
    device = db.device
    od, odp = _out(max(N, 1), np.uint64, device, 2)
    os_, osp = _out(max(N, 1), np.float64, device)
    opts = _Opts()
    lib.asci_default_opts(ct.byref(opts))
    opts.eps_search = float(eps)
    opts.precision = int(precision)
    opts.max_batch_pairs = int(max_batch_pairs)
    opts.max_constraint_level = int(max_constraint_level)
    opts.sort_output = 1 if sort_output else 0
    opts.ctas_per_sm = int(ctas_per_sm)
    if shard is not None:
        opts.shard_index, opts.shard_count = int(shard[0]), int(shard[1])
    st = _Stats()
    n_out = ct.c_size_t(0)
    code = lib.asci_search(db.ptr, cb.ptr, nd, float(E0), ct.byref(ints), int(C), int(N),
                           ct.byref(opts), odp, osp, ct.byref(n_out), ct.byref(st),
                           _stream_ptr(stream, device))
    _check(code, "asci_search")
    m = n_out.value
    return od[:m], os_[:m], (SearchStats._from(st) if return_stats else None)


def pt2(dets, coeffs, E0: float, h1, eri, ecore: float, C: int = None, *, eps: float = 0.0,
        precision: int = FP64, max_batch_pairs: int = 0, max_constraint_level: int = 0,
        stream=None):
    """ASCI-PT2 (Alg. 1, last step): sum over targets i outside psi of
    (sum_j H_ij c_j)^2 / (E0 - H_ii) with the C-determinant core (default: all
    of psi).  Returns (E_PT2, SearchStats)."""
    lib = load()
    keep = []
    db = _dets_buf(dets)
    cb = _as_buf(coeffs, np.float64, "float64")
    keep += [db, cb]
    ints, _ = _ints(h1, eri, ecore, keep)
    nd = int(db.obj.shape[0])
    o = _opts(lib, eps, precision, max_batch_pairs, max_constraint_level, False)
    st = _Stats()
    e = ct.c_double(0.0)
    _check(lib.asci_pt2(db.ptr, cb.ptr, nd, float(E0), ct.byref(ints), int(C or nd), ct.byref(o),
                        ct.byref(e), ct.byref(st), _stream_ptr(stream, db.device)), "asci_pt2")
    return e.value, SearchStats._from(st)


def excitations(h1, eri, ecore, core_dets, core_coeffs, stream=None):
    """Every single and double excitation of each core det with H_ij * c_j (device)."""
    torch = _torch()
    lib = load()
    keep = []
    db = _dets_buf(core_dets)
    cb = _as_buf(core_coeffs, np.float64, "float64")
    if not (db.device and cb.device):
        raise ValueError("excitations() takes CUDA tensors")
    keep += [db, cb]
    ints, _ = _ints(h1, eri, ecore, keep)
    n = ints.norb
    a0 = int(db.obj[0, 0].item()) & ((1 << 64) - 1)
    b0 = int(db.obj[0, 1].item()) & ((1 << 64) - 1)
    na, nb = bin(a0).count("1"), bin(b0).count("1")
    from math import comb
    va, vb = n - na, n - nb
    nexc = na * va + nb * vb + comb(na, 2) * comb(va, 2) + comb(nb, 2) * comb(vb, 2) + na * va * nb * vb
    total = nexc * int(db.obj.shape[0])
    ot = torch.empty((max(total, 1), 2), dtype=torch.int64, device="cuda")
    ov = torch.empty(max(total, 1), dtype=torch.float64, device="cuda")
    n_out = ct.c_size_t(0)
    code = lib.asci_excitations(ct.byref(ints), db.ptr, cb.ptr, int(db.obj.shape[0]),
                                ot.data_ptr(), ov.data_ptr(), total, ct.byref(n_out),
                                _stream_ptr(stream, True))
    _check(code, "asci_excitations")
    return ot[:n_out.value], ov[:n_out.value]


def diagonal(h1, eri, ecore, dets, stream=None):
    """H_ii of each determinant (device)."""
    torch = _torch()
    lib = load()
    keep = []
    db = _dets_buf(dets)
    if not db.device:
        raise ValueError("diagonal() takes CUDA tensors")
    keep.append(db)
    ints, _ = _ints(h1, eri, ecore, keep)
    out = torch.empty(int(db.obj.shape[0]), dtype=torch.float64, device="cuda")
    _check(lib.asci_diagonal(ct.byref(ints), db.ptr, int(db.obj.shape[0]), out.data_ptr(),
                             _stream_ptr(stream, True)), "asci_diagonal")
    return out


def sort_accumulate(keys, values, stream=None):
    """Sort (det, value) pairs on the det and sum per unique det (device)."""
    torch = _torch()
    lib = load()
    kb = _dets_buf(keys)
    vb = _as_buf(values, np.float64, "float64")
    if not (kb.device and vb.device):
        raise ValueError("sort_accumulate() takes CUDA tensors")
    n = int(kb.obj.shape[0])
    ok = torch.empty((max(n, 1), 2), dtype=torch.int64, device="cuda")
    os_ = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    n_out = ct.c_size_t(0)
    _check(lib.asci_sort_accumulate(kb.ptr, vb.ptr, n, ok.data_ptr(), os_.data_ptr(),
                                    ct.byref(n_out), _stream_ptr(stream, True)),
           "asci_sort_accumulate")
    return ok[:n_out.value], os_[:n_out.value]


def _opts(lib, eps, precision, max_batch_pairs, max_constraint_level, sort_output,
          ctas_per_sm=0):
    o = _Opts()
    lib.asci_default_opts(ct.byref(o))
    o.eps_search = float(eps)
    o.precision = int(precision)
    o.max_batch_pairs = int(max_batch_pairs)
    o.max_constraint_level = int(max_constraint_level)
    o.sort_output = 1 if sort_output else 0
    o.ctas_per_sm = int(ctas_per_sm)
    return o


def search_many(systems, *, streams=None, eps: float = 0.0, precision: int = FP64,
                max_batch_pairs: int = 0, max_constraint_level: int = 0,
                sort_output: bool = False, ctas_per_sm: int = 0):
    """Many independent searches (asci_search_many): ``systems`` is a list of
    dicts with keys dets, coeffs, E0, h1, eri, ecore, C, N (arrays as for
    search()).  ``streams`` searches run at a time on their own CUDA streams;
    None picks the count, the batch cap and the CTAs per SM with
    tune_batched().  Returns a list of (dets, scores, stats), each exactly what
    search() returns."""
    lib = load()
    if streams is None:
        t = tune_batched(systems, eps=eps, precision=precision, max_batch_pairs=max_batch_pairs)
        streams, max_batch_pairs = t["streams"], t["max_batch_pairs"]
        ctas_per_sm = t.get("ctas_per_sm", ctas_per_sm)
    keep, probs, outs = [], (_Problem * max(len(systems), 1))(), []
    for i, sy in enumerate(systems):
        db = _dets_buf(sy["dets"])
        cb = _as_buf(sy["coeffs"], np.float64, "float64")
        ints, _ = _ints(sy["h1"], sy["eri"], sy["ecore"], keep)
        N = int(sy["N"])
        od, odp = _out(max(N, 1), np.uint64, db.device, 2)
        os_, osp = _out(max(N, 1), np.float64, db.device)
        n_out, st = ct.c_size_t(0), _Stats()
        keep += [db, cb, ints, n_out, st]
        p = probs[i]
        p.dets, p.coeffs, p.ndets, p.E0 = db.ptr, cb.ptr, int(db.obj.shape[0]), float(sy["E0"])
        p.ints = ct.addressof(ints)
        p.C, p.N = int(sy["C"]), N
        p.out_dets, p.out_scores = odp, osp
        p.out_n, p.stats = ct.addressof(n_out), ct.addressof(st)
        outs.append((od, os_, n_out, st))
    o = _opts(lib, eps, precision, max_batch_pairs, max_constraint_level, sort_output,
              ctas_per_sm)
    code = lib.asci_search_many(ct.addressof(probs), len(systems), ct.byref(o), int(streams))
    _check(code, "asci_search_many")
    if len(systems) and outs[0][0].__class__.__module__.startswith("torch"):
        _torch().cuda.synchronize()
    return [(od[:n.value], os_[:n.value], SearchStats._from(st)) for od, os_, n, st in outs]


_TUNED = {}


def tune_batched(systems, streams=(1, 2, 4, 8, 16, 32), batch_caps=(0, 1 << 22, 1 << 20),
                 ctas=(0, 2, 1), sample: int = 64, **kw):
    """The project's autotuner for batched searches: a grid search over the
    number of concurrent streams, the constraint-batch cap (pairs per batch;
    0 = sized from free memory) and the launch shape of the persistent kernels
    (CTAs per SM; 0 = as many as fit: fewer leave the GPU to the other
    streams' searches), keeping the point that gives the most searches per
    second on a sample of the batch.  Cached per batch signature (whether the
    batch exceeds the sample, the largest orbital count, the precision).
    Returns {"streams": k, "max_batch_pairs": b, "ctas_per_sm": c}.  A given
    max_batch_pairs or ctas_per_sm in kw fixes that coordinate."""
    import time
    fixed = int(kw.pop("max_batch_pairs", 0) or 0)
    fixed_ctas = kw.pop("ctas_per_sm", None)
    if not systems:
        return {"streams": 1, "max_batch_pairs": fixed, "ctas_per_sm": int(fixed_ctas or 0)}
    norb = max(int(round(np.sqrt(np.prod(np.shape(sy["h1"]))))) for sy in systems)
    caps = (fixed,) if fixed else tuple(batch_caps)
    shapes = (int(fixed_ctas),) if fixed_ctas is not None else tuple(ctas)
    sig = (len(systems) >= sample, norb, kw.get("precision", FP64), caps, shapes)
    if sig in _TUNED:
        return dict(_TUNED[sig])
    sub = systems[:sample]
    best, best_rate = {"streams": 1, "max_batch_pairs": caps[0], "ctas_per_sm": shapes[0]}, -1.0
    search_many(sub[:2], streams=1, max_batch_pairs=caps[0], ctas_per_sm=shapes[0],
                **kw)  # warm caches and the pool
    for c in shapes:
        for b in caps:
            for k in streams:
                if k > len(sub):
                    break
                t0 = time.perf_counter()
                search_many(sub, streams=k, max_batch_pairs=b, ctas_per_sm=c, **kw)
                rate = len(sub) / (time.perf_counter() - t0)
                if rate > best_rate:
                    best, best_rate = {"streams": k, "max_batch_pairs": b, "ctas_per_sm": c}, rate
    _TUNED[sig] = dict(best)
    return best


def tune_streams(systems, candidates=(1, 2, 4, 8, 16, 32), sample: int = 64, **kw):
    """The stream count of tune_batched with the batch cap fixed to kw's
    max_batch_pairs (default 0: sized from free memory)."""
    cap = int(kw.pop("max_batch_pairs", 0) or 0)
    return tune_batched(systems, streams=candidates, batch_caps=(cap,), sample=sample,
                        **kw)["streams"]


def shard_assign(weights, shards: int, initial_loads=None):
    """Alg. 3's greedy placement of classes of the given weights onto shards
    (heaviest first, each to the least-loaded shard; host computation)."""
    lib = load()
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.uint64))
    out = np.empty(len(w), dtype=np.int32)
    init = None
    if initial_loads is not None:
        init = np.ascontiguousarray(np.asarray(initial_loads, dtype=np.uint64))
        if len(init) != shards:
            raise ValueError("initial_loads needs one entry per shard")
    _check(lib.asci_shard_assign(w.ctypes.data if len(w) else None, len(w), int(shards),
                                 init.ctypes.data if init is not None else None,
                                 out.ctypes.data if len(w) else None), "asci_shard_assign")
    return out


def gather_candidates(keys, scores, group=None):
    """All ranks' candidates, concatenated in rank order, on every rank.

    keys: (m, 2) int64 tensor, scores: (m,) float64 tensor, m may differ by
    rank.  Uses torch.distributed (NCCL for CUDA tensors, gloo for CPU ones):
    the counts first, then the padded lists.
    """
    torch = _torch()
    import torch.distributed as dist
    W = dist.get_world_size(group)
    dev = keys.device
    m = torch.tensor([keys.shape[0]], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(m) for _ in range(W)]
    dist.all_gather(counts, m, group=group)
    counts = [int(c.item()) for c in counts]
    mx = max(counts) if counts else 0
    kp = torch.zeros((mx, 2), dtype=torch.int64, device=dev)
    sp = torch.zeros(mx, dtype=torch.float64, device=dev)
    kp[:keys.shape[0]] = keys
    sp[:scores.shape[0]] = scores
    kl = [torch.empty_like(kp) for _ in range(W)]
    sl = [torch.empty_like(sp) for _ in range(W)]
    dist.all_gather(kl, kp, group=group)
    dist.all_gather(sl, sp, group=group)
    return (torch.cat([k[:c] for k, c in zip(kl, counts)]),
            torch.cat([v[:c] for v, c in zip(sl, counts)]))


def constraint_classes(dets, coeffs, h1, eri, ecore: float, C: int, level: int, stream=None):
    """Pair counts of the constraint classes of one level (Sec. 2.2: targets
    sharing their `level` highest occupied alpha orbitals), in ascending
    order of the classes' alpha strings: numpy uint64 array (a size query,
    then the call)."""
    lib = load()
    keep = []
    db = _dets_buf(dets)
    cb = _as_buf(coeffs, np.float64, "float64")
    keep += [db, cb]
    ints, _ = _ints(h1, eri, ecore, keep)
    n_out = ct.c_size_t(0)
    sp = _stream_ptr(stream, db.device)
    args = (db.ptr, cb.ptr, int(db.obj.shape[0]), ct.byref(ints), int(C), int(level))
    _check(lib.asci_constraint_classes(*args, None, 0, ct.byref(n_out), sp),
           "asci_constraint_classes")
    out = np.zeros(max(n_out.value, 1), dtype=np.uint64)
    _check(lib.asci_constraint_classes(*args, out.ctypes.data, out.size, ct.byref(n_out), sp),
           "asci_constraint_classes")
    return out[:n_out.value]


def select_histogram(keys, scores, digit: int, prefix, mask, stream=None):
    """Histogram (numpy uint64[256]) of byte `digit` of the rank word
    (~bits(|score|), key) over the entries matching prefix on mask (device)."""
    lib = load()
    kb = _dets_buf(keys)
    sb = _as_buf(scores, np.float64, "float64")
    n = int(kb.obj.shape[0])
    pre = np.ascontiguousarray(prefix, dtype=np.uint64)
    msk = np.ascontiguousarray(mask, dtype=np.uint64)
    h = np.zeros(256, dtype=np.uint64)
    _check(lib.asci_select_histogram(kb.ptr if n else None, sb.ptr if n else None, n, int(digit),
                                     pre.ctypes.data, msk.ctypes.data, h.ctypes.data,
                                     _stream_ptr(stream, kb.device)), "asci_select_histogram")
    return h


def select_below(keys, scores, threshold, stream=None):
    """The entries whose rank word is at most threshold ({hi, lo}) (device)."""
    torch = _torch()
    lib = load()
    kb = _dets_buf(keys)
    sb = _as_buf(scores, np.float64, "float64")
    n = int(kb.obj.shape[0])
    ok = torch.empty((max(n, 1), 2), dtype=torch.int64, device="cuda")
    os_ = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    thr = np.ascontiguousarray(threshold, dtype=np.uint64)
    n_out = ct.c_size_t(0)
    _check(lib.asci_select_below(kb.ptr if n else None, sb.ptr if n else None, n, thr.ctypes.data,
                                 ok.data_ptr(), os_.data_ptr(), ct.byref(n_out),
                                 _stream_ptr(stream, True)), "asci_select_below")
    return ok[:n_out.value], os_[:n_out.value]


def distributed_topn(keys, scores, N: int, group=None, hist_fn=None, below_fn=None):
    """The global top N (|score| descending, key ascending) of candidates
    spread over the ranks of a torch.distributed group, the role of Alg. 4:
    the N-th rank word is found byte by byte from the most significant end,
    each byte by an all-reduce of the ranks' 256-bin histograms (2 KB), then
    each rank keeps its entries at or below it and the winners, N in all, are
    gathered to every rank.  hist_fn(digit, prefix, mask) and
    below_fn(threshold) are the local steps (the library's kernels by
    default).  Returns (keys, scores) of the global top N on every rank."""
    torch = _torch()
    import torch.distributed as dist
    lib = load()
    hist_fn = hist_fn or (lambda d, p, m: select_histogram(keys, scores, d, p, m))
    below_fn = below_fn or (lambda t: select_below(keys, scores, t))
    dev = keys.device
    total = torch.tensor([keys.shape[0]], dtype=torch.int64, device=dev)
    dist.all_reduce(total, group=group)
    st = _SelectState()
    _check(lib.asci_select_begin(int(total.item()), int(N), ct.byref(st)), "asci_select_begin")
    while not st.done:
        h = torch.tensor(np.asarray(hist_fn(st.digit, list(st.prefix), list(st.mask)))
                         .astype(np.int64), device=dev)
        dist.all_reduce(h, group=group)
        hh = np.ascontiguousarray(h.cpu().numpy().astype(np.uint64))
        _check(lib.asci_select_step(ct.byref(st), hh.ctypes.data), "asci_select_step")
    wk, ws = below_fn(list(st.threshold))
    return gather_candidates(wk, ws, group)


def sharded_search(dets, coeffs, E0: float, h1, eri, ecore: float, C: int, N: int, *,
                   group=None, **kw):
    """One search sharded over the ranks of a torch.distributed group (one GPU
    per rank): each rank searches its shard of the target alpha classes and
    keeps its top N; the global top N of the union is then selected across the
    ranks (distributed_topn) without gathering the shards' lists (the shards
    partition the targets, so this is the unsharded result).  Returns (dets,
    scores, local stats) with the global top N on every rank."""
    import torch.distributed as dist
    r, W = dist.get_rank(group), dist.get_world_size(group)
    od, osc, st = search(dets, coeffs, E0, h1, eri, ecore, C, N, shard=(r, W), **kw)
    gk, gs = distributed_topn(od, osc, N, group)
    return gk, gs, st


def select_topn(keys, scores, N: int, stream=None):
    """Top-N by |score|, ties by key ascending (device)."""
    torch = _torch()
    lib = load()
    kb = _dets_buf(keys)
    sb = _as_buf(scores, np.float64, "float64")
    if not (kb.device and sb.device):
        raise ValueError("select_topn() takes CUDA tensors")
    n = int(kb.obj.shape[0])
    m = max(min(n, N), 1)
    ok = torch.empty((m, 2), dtype=torch.int64, device="cuda")
    os_ = torch.empty(m, dtype=torch.float64, device="cuda")
    n_out = ct.c_size_t(0)
    _check(lib.asci_select_topn(kb.ptr, sb.ptr, n, int(N), ok.data_ptr(), os_.data_ptr(),
                                ct.byref(n_out), _stream_ptr(stream, True)), "asci_select_topn")
    return ok[:n_out.value], os_[:n_out.value]


# ------------------------- the variational step ----------------------------

def hamiltonian(dets, h1, eri, ecore, stream=None):
    """H restricted to the determinant list (Sec. 2.3), CSR on the device:
    (row_ptr int64[n+1], col int32[nnz], val float64[nnz]).  Two calls of
    asci_hamiltonian: the size query, then the fill."""
    torch = _torch()
    lib = load()
    keep = []
    db = _dets_buf(dets)
    keep.append(db)
    ints, _ = _ints(h1, eri, ecore, keep)
    n = int(db.obj.shape[0])
    rp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    nnz = ct.c_size_t(0)
    sp = _stream_ptr(stream, True)
    _check(lib.asci_hamiltonian(db.ptr, n, ct.byref(ints), rp.data_ptr(), None, None, 0,
                                ct.byref(nnz), sp), "asci_hamiltonian")
    col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device="cuda")
    val = torch.empty(max(nnz.value, 1), dtype=torch.float64, device="cuda")
    _check(lib.asci_hamiltonian(db.ptr, n, ct.byref(ints), rp.data_ptr(), col.data_ptr(),
                                val.data_ptr(), nnz.value, ct.byref(nnz), sp), "asci_hamiltonian")
    return rp, col[:nnz.value], val[:nnz.value]


def spmv(H, x, stream=None):
    """y = H x for H = (row_ptr, col, val) from hamiltonian() (device)."""
    torch = _torch()
    lib = load()
    rp, col, val = H
    n = rp.shape[0] - 1
    xb = _as_buf(x, np.float64, "float64")
    if not xb.device:
        raise ValueError("spmv() takes CUDA tensors")
    y = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    _check(lib.asci_spmv(rp.data_ptr(), col.data_ptr(), val.data_ptr(), n, xb.ptr, y.data_ptr(),
                         _stream_ptr(stream, True)), "asci_spmv")
    return y[:n]


def davidson(H, guess=None, *, max_subspace: int = 16, max_iter: int = 300, tol: float = 1e-8,
             stream=None):
    """Lowest eigenpair of H = (row_ptr, col, val) by Davidson (Alg. 5).
    Returns (energy, vector (device), products with H, residual norm)."""
    torch = _torch()
    lib = load()
    rp, col, val = H
    n = rp.shape[0] - 1
    gp = None
    if guess is not None:
        gb = _as_buf(guess, np.float64, "float64")
        if not gb.device:
            raise ValueError("davidson() takes a CUDA guess")
        guess, gp = gb.obj, gb.ptr
    o = _DavOpts(int(max_subspace), int(max_iter), float(tol))
    vec = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    e, it, res = ct.c_double(0.0), ct.c_int32(0), ct.c_double(0.0)
    _check(lib.asci_davidson(rp.data_ptr(), col.data_ptr(), val.data_ptr(), n, gp, ct.byref(o),
                             ct.byref(e), vec.data_ptr(), ct.byref(it), ct.byref(res),
                             _stream_ptr(stream, True)), "asci_davidson")
    return e.value, vec[:n], it.value, res.value


def asci_loop(dets, coeffs, h1, eri, ecore, *, ncdets: int, ntdets: int, max_steps: int = 8,
              etol: float = 1e-6, eps: float = 0.0, precision: int = FP64,
              max_batch_pairs: int = 0, max_subspace: int = 16, max_iter: int = 300,
              tol: float = 1e-8, stream=None):
    """The ASCI loop (Alg. 1): search, keep the ntdets largest of |c| and |S|,
    build H on that space, Davidson; repeat.  Returns (dets, coeffs, energy,
    LoopStats); outputs live where ``dets`` lives."""
    lib = load()
    keep = []
    db = _dets_buf(dets)
    cb = _as_buf(coeffs, np.float64, "float64")
    keep += [db, cb]
    ints, _ = _ints(h1, eri, ecore, keep)
    o = _LoopOpts()
    lib.asci_default_loop_opts(ct.byref(o))
    o.ncdets, o.ntdets, o.max_steps, o.etol = int(ncdets), int(ntdets), int(max_steps), float(etol)
    o.search = _opts(lib, eps, precision, max_batch_pairs, 0, False)
    o.davidson = _DavOpts(int(max_subspace), int(max_iter), float(tol))
    cap = int(ntdets)
    od, odp = _out(max(cap, 1), np.uint64, db.device, 2)
    oc, ocp = _out(max(cap, 1), np.float64, db.device)
    n_out, energy, st = ct.c_size_t(0), ct.c_double(0.0), _LoopStats()
    _check(lib.asci_loop(db.ptr, cb.ptr, int(db.obj.shape[0]), ct.byref(ints), ct.byref(o), odp,
                         ocp, cap, ct.byref(n_out), ct.byref(energy), ct.byref(st),
                         _stream_ptr(stream, db.device)), "asci_loop")
    m = n_out.value
    return od[:m], oc[:m], energy.value, LoopStats._from(st)
