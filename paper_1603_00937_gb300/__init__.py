"""Python binding of libgbe: graph-partitioned SP2 density matrices on GB300.

Argument marshalling only -- every step of the computation runs in the CUDA kernels of
libgbe.so (built in-tree by ``build.py``).  Names follow the C ABI in include/gbe.h.
Device arrays are torch CUDA tensors (PyTorch supplies device memory and streams);
NumPy arrays are passed as host buffers where the ABI accepts them.

There is no CPU fallback: importing works without a GPU, but creating a context fails
loudly when the library or a usable sm_103 device is missing.

Example (one density matrix of the 32^3 lattice; every step runs in the library's kernels)::

    import torch, synth
    import paper_1603_00937_gb300 as gbe

    w = synth.lattice(32, seed=0)                                   # 32^3 sites, N = 32,768
    ctx = gbe.Context(0)
    st = gbe.sites(torch.from_numpy(w["pos"]).cuda(), torch.from_numpy(w["onsite"]).cuda(), w["box"])
    H = gbe.build_hamiltonian(ctx, st)                              # device CSR H
    S = gbe.build_graph(ctx, H.csr(), gbe.GRAPH_H2_THRESH, thresh=0.15)     # Eq. 2 on H^2
    parts = gbe.partition(ctx, S, gbe.PART_SPATIAL_CELLS, ncell=(8, 8, 8), site_struct=st)
    X, rep = gbe.sp2_submatrices(ctx, H.csr(), parts, gbe.sp2_params(16384, prec=gbe.PREC_FP16X6))
    n, width = gbe.assemble_width(ctx, X, parts)
    col = torch.empty((n, width), dtype=torch.int32, device="cuda")
    val = torch.empty((n, width), dtype=torch.float64, device="cuda")
    gbe.assemble_D(ctx, X, parts, col, val)                         # row i of the ELL = column i of D (Eq. 6)
    print(rep["iters"], rep["stop"])
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbe.so")

GBE_OK, GBE_EINVAL, GBE_ENOMEM, GBE_ECUDA, GBE_ETIMEOUT = 0, -1, -2, -3, -4
GBE_ENOCONV, GBE_ENUMERIC, GBE_ECAPACITY, GBE_ENODEV, GBE_EPEER = -5, -6, -7, -8, -9

GRAPH_H2_THRESH, GRAPH_D_THRESH, GRAPH_EQ8_SYMBOLIC, GRAPH_HK_PATTERN, GRAPH_MLP = 0, 1, 2, 3, 4
PART_SPATIAL_CELLS, PART_INDEX_BLOCKS = 0, 1
PREC_FP64, PREC_FP16X6, PREC_BF16X3, PREC_FP64TC = 0, 1, 2, 3
BRANCH_GLOBAL_TRACE, BRANCH_REPLAY = 0, 1
SCHED_ROUND_ROBIN, SCHED_BALANCED_RANGES = 0, 1
SCHED_NAMES = {0: "round_robin", 1: "balanced_ranges"}
TUNE_MAX = 16
STOP_NAMES = {0: "none", 1: "tol", 2: "stall", 3: "nmax", 4: "replay", 5: "error"}
SEQ_MAX = 256

# Every entry point declared in include/gbe.h (checked by the CPU test suite).
EXPORTS = [
    "gbe_create", "gbe_destroy", "gbe_set_stream", "gbe_set_profiling", "gbe_set_graph_launch", "gbe_device_sm_count", "gbe_strerror",
    "gbe_last_error_message", "gbe_build_hamiltonian", "gbe_hamiltonian_csr", "gbe_free_hamiltonian",
    "gbe_build_graph", "gbe_graph_size", "gbe_graph_export", "gbe_free_graph", "gbe_partition",
    "gbe_parts_info", "gbe_parts_export", "gbe_parts_import", "gbe_free_parts", "gbe_subs_create",
    "gbe_free_subs", "gbe_sp2_run", "gbe_sp2_report_get", "gbe_sp2_replay_batched", "gbe_sp2_submatrices", "gbe_assemble_D",
    "gbe_subs_export", "gbe_gershgorin_noalloc", "gbe_pairs_build", "gbe_pairs_info", "gbe_pairs_export", "gbe_pairs_device",
    "gbe_free_pairs", "gbe_mlp_create", "gbe_mlp_param_count", "gbe_mlp_set_params", "gbe_mlp_get_params",
    "gbe_mlp_forward", "gbe_mlp_gradient", "gbe_mlp_adam_step", "gbe_mlp_train", "gbe_mlp_labels", "gbe_free_mlp",
    "gbe_sp2_gap_estimate", "gbe_sp2_sequence", "gbe_fermi_coefficients", "gbe_foe_run", "gbe_foe_report_get",
    "gbe_subs_get_config", "gbe_subs_set_config", "gbe_sp2_autotune", "gbe_partition_autotune",
    "gbe_shard_assign", "gbe_parts_shard",
]

# gbe_exchange_fn: int (*)(void* user, double* buf, int64_t count, void* stream)
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p)


class GbeError(RuntimeError):
    def __init__(self, code, where, detail):
        super().__init__("%s failed: %s (%d): %s" % (where, _strerror(code), code, detail))
        self.code = code


class Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("on_device", ctypes.c_int)]


class Ell(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("width", ctypes.c_int64), ("col", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("on_device", ctypes.c_int)]


class Sites(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("pos", ctypes.c_void_p), ("onsite", ctypes.c_void_p),
                ("box", ctypes.c_double * 3), ("on_device", ctypes.c_int)]


class TbModel(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("rcut", ctypes.c_double), ("decay", ctypes.c_double),
                ("hop", ctypes.c_double)]


class GraphParams(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("thresh", ctypes.c_double), ("k", ctypes.c_int),
                ("D_prev", ctypes.c_void_p), ("sites", ctypes.c_void_p), ("mlp", ctypes.c_void_p),
                ("rcand", ctypes.c_double), ("logit_cut", ctypes.c_double)]


class PartitionParams(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("ncell", ctypes.c_int * 3), ("sites", ctypes.c_void_p),
                ("core_size", ctypes.c_int), ("max_sub", ctypes.c_int)]


class Sp2Params(ctypes.Structure):
    _fields_ = [("n_occ", ctypes.c_double), ("idem_tol", ctypes.c_double), ("n_min", ctypes.c_int),
                ("n_max", ctypes.c_int), ("prec", ctypes.c_int), ("fp64_tail", ctypes.c_int),
                ("tail_switch", ctypes.c_double), ("branch_mode", ctypes.c_int),
                ("seq_in", ctypes.c_void_p), ("seq_len", ctypes.c_int), ("eps_given", ctypes.c_int),
                ("eps_min", ctypes.c_double), ("eps_max", ctypes.c_double), ("timeout_ms", ctypes.c_double),
                ("exchange", EXCHANGE_FN), ("exchange_user", ctypes.c_void_p)]


class Sp2Report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("fp64_iters", ctypes.c_int), ("stop_reason", ctypes.c_int),
                ("converged", ctypes.c_int), ("status", ctypes.c_int), ("eps_min", ctypes.c_double),
                ("eps_max", ctypes.c_double), ("trace", ctypes.c_double), ("idem_err", ctypes.c_double),
                ("seq", ctypes.c_uint8 * SEQ_MAX), ("t1", ctypes.c_double * (SEQ_MAX + 1)),
                ("t2", ctypes.c_double * (SEQ_MAX + 1)), ("ms_gather", ctypes.c_float),
                ("ms_sp2", ctypes.c_float), ("mma_flops", ctypes.c_double), ("alg_flops", ctypes.c_double),
                ("ms_tc", ctypes.c_float), ("ms_fp64", ctypes.c_float), ("n_tc", ctypes.c_int),
                ("n_fp64", ctypes.c_int), ("fp64_flops", ctypes.c_double)]

    def as_dict(self):
        n = self.iters
        return dict(iters=n, fp64_iters=self.fp64_iters, stop=STOP_NAMES.get(self.stop_reason, "?"),
                    converged=bool(self.converged), status=self.status, eps=(self.eps_min, self.eps_max),
                    trace=self.trace, idem_err=self.idem_err, seq=list(self.seq[:n]),
                    t1=list(self.t1[:n + 1]), t2=list(self.t2[:n + 1]), ms_gather=self.ms_gather,
                    ms_sp2=self.ms_sp2, mma_flops=self.mma_flops, alg_flops=self.alg_flops,
                    ms_tc=self.ms_tc, n_tc=self.n_tc, ms_fp64=self.ms_fp64, n_fp64=self.n_fp64,
                    fp64_flops=self.fp64_flops)


class TcConfig(ctypes.Structure):
    _fields_ = [("stages", ctypes.c_int), ("schedule", ctypes.c_int), ("kchunk", ctypes.c_int)]


class TuneReport(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("cand", TcConfig * TUNE_MAX), ("ms", ctypes.c_float * TUNE_MAX),
                ("best", ctypes.c_int), ("iters", ctypes.c_int), ("cached", ctypes.c_int)]

    def as_dict(self):
        cands = [dict(kchunk=self.cand[i].kchunk or 32, stages=self.cand[i].stages,
                      schedule=SCHED_NAMES.get(self.cand[i].schedule, "?"), ms_per_run=self.ms[i])
                 for i in range(self.n)]
        return dict(candidates=cands, best=cands[self.best] if self.n else None, iters=self.iters,
                    cached=bool(self.cached))


_lib = None


def load_library(path=LIB_PATH):
    """Load libgbe.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libgbe.so not found at %s: run paper_1603_00937_gb300/build.py "
                           "(or __graft_entry__.build()) first; there is no CPU fallback" % path)
    lib = ctypes.CDLL(path)
    P, I64, I32, D, C = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_char_p
    sig = {
        "gbe_create": (I32, [P, I32, P]), "gbe_destroy": (I32, [P]), "gbe_set_stream": (I32, [P, P]),
        "gbe_device_sm_count": (I32, [P]), "gbe_set_profiling": (I32, [P, I32]), "gbe_set_graph_launch": (I32, [P, I32]), "gbe_strerror": (C, [I32]), "gbe_last_error_message": (C, []),
        "gbe_build_hamiltonian": (I32, [P, P, P, P]), "gbe_hamiltonian_csr": (I32, [P, P]),
        "gbe_free_hamiltonian": (I32, [P]), "gbe_build_graph": (I32, [P, P, P, P]),
        "gbe_graph_size": (I32, [P, P, P, P]), "gbe_graph_export": (I32, [P, P, P, P]),
        "gbe_free_graph": (I32, [P]), "gbe_partition": (I32, [P, P, P, P]),
        "gbe_parts_info": (I32, [P, P, P, P]), "gbe_parts_export": (I32, [P, P, P, P, P]),
        "gbe_parts_import": (I32, [P, I64, I64, P, P, P, P]), "gbe_free_parts": (I32, [P]),
        "gbe_subs_create": (I32, [P, P, I32, P]), "gbe_free_subs": (I32, [P]),
        "gbe_sp2_run": (I32, [P, P, P, P, P]), "gbe_sp2_report_get": (I32, [P, P, P]),
        "gbe_sp2_submatrices": (I32, [P, P, P, P, P, P]), "gbe_assemble_D": (I32, [P, P, P, D, P]),
        "gbe_sp2_replay_batched": (I32, [P, P, P, P, ctypes.c_int64, D, P, P]),
        "gbe_subs_export": (I32, [P, P, I64, P]), "gbe_gershgorin_noalloc": (I32, [P, P, P]),
        "gbe_pairs_build": (I32, [P, P, P, D, P]), "gbe_pairs_info": (I32, [P, P, P]),
        "gbe_pairs_export": (I32, [P, P, P, P, P]), "gbe_free_pairs": (I32, [P]),
        "gbe_pairs_device": (I32, [P, P, P, P]),
        "gbe_mlp_create": (I32, [P, I32, P]), "gbe_mlp_param_count": (I32, [P]),
        "gbe_mlp_set_params": (I32, [P, P, P]), "gbe_mlp_get_params": (I32, [P, P, P]),
        "gbe_mlp_forward": (I32, [P, P, P, P]), "gbe_mlp_gradient": (I32, [P, P, P, P, P, P]),
        "gbe_mlp_adam_step": (I32, [P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
        "gbe_mlp_train": (I32, [P, P, P, P, I32, ctypes.c_float, P]), "gbe_free_mlp": (I32, [P]),
        "gbe_mlp_labels": (I32, [P, P, P, D, P]),
        "gbe_sp2_gap_estimate": (I32, [P, D, D, D, P, P]), "gbe_sp2_sequence": (I32, [D, D, D, D, D, I32, P, P]),
        "gbe_fermi_coefficients": (I32, [D, D, D, D, I32, P]), "gbe_foe_run": (I32, [P, P, P, P, P]),
        "gbe_foe_report_get": (I32, [P, P, P]),
        "gbe_subs_get_config": (I32, [P, P]), "gbe_subs_set_config": (I32, [P, P, P]),
        "gbe_sp2_autotune": (I32, [P, P, P, P, P, I32, P]),
        "gbe_partition_autotune": (I32, [P, P, P, I32, P, I32, P, P, P]),
        "gbe_shard_assign": (I32, [I64, P, I32, P, P]), "gbe_parts_shard": (I32, [P, P, P, I32, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _strerror(code):
    try:
        return load_library().gbe_strerror(code).decode()
    except Exception:
        return "error"


def check(code, where):
    if code != GBE_OK:
        detail = load_library().gbe_last_error_message().decode(errors="replace")
        raise GbeError(code, where, detail)
    return code


def _ptr(a):
    """Raw pointer of a torch tensor (device or host) or a contiguous NumPy array."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()


def _is_device(a):
    return (not isinstance(a, np.ndarray)) and getattr(a, "is_cuda", False)


def csr(n, rowptr, col, val):
    """gbe_csr over (int64 rowptr, int32 col, float64 val), all torch-CUDA or all NumPy."""
    dev = _is_device(rowptr)
    keep = (rowptr, col, val)
    c = Csr(n, int(col.shape[0]), _ptr(rowptr), _ptr(col), _ptr(val), 1 if dev else 0)
    c._keep = keep
    return c


class Context:
    def __init__(self, device=0, stream=None):
        lib = load_library()
        self._h = ctypes.c_void_p()
        s = ctypes.c_void_p(stream) if stream is not None else None
        check(lib.gbe_create(ctypes.byref(self._h), device, s), "gbe_create")

    @property
    def handle(self):
        return self._h

    def set_profiling(self, on=True):
        check(load_library().gbe_set_profiling(self._h, 1 if on else 0), "gbe_set_profiling")

    def set_graph_launch(self, on=True):
        check(load_library().gbe_set_graph_launch(self._h, 1 if on else 0), "gbe_set_graph_launch")

    def set_stream(self, stream):
        check(load_library().gbe_set_stream(self._h, ctypes.c_void_p(stream)), "gbe_set_stream")

    @property
    def sm_count(self):
        return load_library().gbe_device_sm_count(self._h)

    def close(self):
        if self._h:
            load_library().gbe_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Owned:
    _free = None

    def __init__(self, ctx, h):
        self.ctx, self._h = ctx, h

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            getattr(load_library(), self._free)(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hamiltonian(_Owned):
    _free = "gbe_free_hamiltonian"

    def csr(self):
        v = Csr()
        check(load_library().gbe_hamiltonian_csr(self._h, ctypes.byref(v)), "gbe_hamiltonian_csr")
        v._keep = self
        return v


class Graph(_Owned):
    _free = "gbe_free_graph"

    def size(self):
        n, nnz = ctypes.c_int64(), ctypes.c_int64()
        check(load_library().gbe_graph_size(self.ctx.handle, self._h, ctypes.byref(n), ctypes.byref(nnz)),
              "gbe_graph_size")
        return n.value, nnz.value

    def export(self):
        n, nnz = self.size()
        rowptr = np.zeros(n + 1, dtype=np.int64)
        col = np.zeros(max(nnz, 1), dtype=np.int32)
        check(load_library().gbe_graph_export(self.ctx.handle, self._h, _ptr(rowptr), _ptr(col)),
              "gbe_graph_export")
        return rowptr, col[:nnz]


class Parts(_Owned):
    _free = "gbe_free_parts"

    def info(self):
        P, total, max_m = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(load_library().gbe_parts_info(self._h, ctypes.byref(P), ctypes.byref(total), ctypes.byref(max_m)),
              "gbe_parts_info")
        return P.value, total.value, max_m.value

    def export(self):
        """(core_count[P], sub_ptr[P+1], sub_idx[total]) as NumPy arrays."""
        P, total, _ = self.info()
        cc = np.zeros(P, dtype=np.int32)
        sp = np.zeros(P + 1, dtype=np.int64)
        si = np.zeros(total, dtype=np.int32)
        check(load_library().gbe_parts_export(self.ctx.handle, self._h, _ptr(cc), _ptr(sp), _ptr(si)),
              "gbe_parts_export")
        return cc, sp, si


class Subs(_Owned):
    _free = "gbe_free_subs"

    def export(self, s, m):
        out = np.zeros((m, m), dtype=np.float64)
        check(load_library().gbe_subs_export(self.ctx.handle, self._h, int(s), _ptr(out)), "gbe_subs_export")
        return out


def sites(pos, onsite, box):
    dev = _is_device(pos)
    s = Sites(int(pos.shape[0]), _ptr(pos), _ptr(onsite), (ctypes.c_double * 3)(*[float(b) for b in box]),
              1 if dev else 0)
    s._keep = (pos, onsite)
    return s


def tb_model(a=1.0, rcut=2.5, decay=0.3, hop=-1.0):
    return TbModel(a, rcut, decay, hop)


def build_hamiltonian(ctx, site_struct, model=None):
    h = ctypes.c_void_p()
    model = model or tb_model()
    check(load_library().gbe_build_hamiltonian(ctx.handle, ctypes.byref(site_struct), ctypes.byref(model),
                                               ctypes.byref(h)), "gbe_build_hamiltonian")
    return Hamiltonian(ctx, h)


def build_graph(ctx, H, mode, thresh=0.0, k=1, D_prev=None, site_struct=None, mlp=None, rcand=0.0,
                logit_cut=0.0):
    p = GraphParams(mode, thresh, k, ctypes.cast(ctypes.pointer(D_prev), ctypes.c_void_p) if D_prev is not None else None,
                    ctypes.cast(ctypes.pointer(site_struct), ctypes.c_void_p) if site_struct is not None else None,
                    mlp.handle if mlp is not None else None, rcand, logit_cut)
    g = ctypes.c_void_p()
    check(load_library().gbe_build_graph(ctx.handle, ctypes.byref(H), ctypes.byref(p), ctypes.byref(g)),
          "gbe_build_graph")
    return Graph(ctx, g)


def partition(ctx, S, mode=PART_SPATIAL_CELLS, ncell=(1, 1, 1), site_struct=None, core_size=0, max_sub=0):
    p = PartitionParams(mode, (ctypes.c_int * 3)(*ncell),
                        ctypes.cast(ctypes.pointer(site_struct), ctypes.c_void_p) if site_struct is not None else None,
                        core_size, max_sub)
    h = ctypes.c_void_p()
    check(load_library().gbe_partition(ctx.handle, S.handle, ctypes.byref(p), ctypes.byref(h)), "gbe_partition")
    return Parts(ctx, h)


def partition_autotune(ctx, S, candidates, prec=PREC_FP16X6, mode=PART_SPATIAL_CELLS, site_struct=None, max_sub=0):
    """Cost-driven partition size: candidates are ncell triples (spatial cells) or core sizes
    (index blocks).  Returns (Parts of the cheapest, index of it, per-candidate costs)."""
    cand = np.zeros((len(candidates), 3), dtype=np.int32)
    for i, c in enumerate(candidates):
        cand[i, :len(np.atleast_1d(c))] = np.atleast_1d(c)
    pp = PartitionParams(mode, (ctypes.c_int * 3)(1, 1, 1),
                         ctypes.cast(ctypes.pointer(site_struct), ctypes.c_void_p) if site_struct is not None else None,
                         0, max_sub)
    cost = np.zeros(len(candidates), dtype=np.float64)
    best = ctypes.c_int()
    h = ctypes.c_void_p()
    check(load_library().gbe_partition_autotune(ctx.handle, S.handle, ctypes.byref(pp), prec, _ptr(cand), len(cand),
                                                _ptr(cost), ctypes.byref(best), ctypes.byref(h)), "gbe_partition_autotune")
    return Parts(ctx, h), best.value, cost


def parts_import(ctx, n, core_count, sub_ptr, sub_idx):
    cc = np.ascontiguousarray(core_count, dtype=np.int32)
    sp = np.ascontiguousarray(sub_ptr, dtype=np.int64)
    si = np.ascontiguousarray(sub_idx, dtype=np.int32)
    h = ctypes.c_void_p()
    check(load_library().gbe_parts_import(ctx.handle, int(n), len(cc), _ptr(cc), _ptr(sp), _ptr(si),
                                          ctypes.byref(h)), "gbe_parts_import")
    return Parts(ctx, h)


def sp2_params(n_occ, prec=PREC_FP64, idem_tol=1e-10, n_min=10, n_max=100, fp64_tail=0, tail_switch=0.0,
               seq=None, eps=None, timeout_ms=0.0, exchange=None):
    """gbe_sp2_params.  exchange: for a sharded run (parts from parts_shard), a callable
    (buf_ptr, count, stream_ptr) that replaces the `count` doubles at the device address
    buf_ptr by their sum over all ranks, ordered on the stream (see dist_exchange)."""
    buf = None
    if seq is not None:
        buf = np.ascontiguousarray(np.asarray(seq, dtype=np.uint8))
    p = Sp2Params(float(n_occ), idem_tol, n_min, n_max, prec, fp64_tail, tail_switch,
                  BRANCH_REPLAY if seq is not None else BRANCH_GLOBAL_TRACE,
                  _ptr(buf) if buf is not None and len(buf) else None, 0 if buf is None else len(buf),
                  1 if eps is not None else 0, eps[0] if eps is not None else 0.0,
                  eps[1] if eps is not None else 0.0, timeout_ms)
    if buf is not None and len(buf) == 0:
        p.seq_in = ctypes.cast(ctypes.create_string_buffer(1), ctypes.c_void_p)
    cb = None
    if exchange is not None:
        def _cb(user, ptr, count, stream):
            try:
                exchange(ptr, count, stream)
                return 0
            except Exception:
                return 1
        cb = EXCHANGE_FN(_cb)
        p.exchange = cb
    p._keep = (buf, cb)
    return p


def shard_assign(sub_ptr, world):
    """(owner[P], load[world]): subgraphs dealt to ranks by greedy longest-processing-time on
    m_s^3 (gbe_shard_assign; host only)."""
    sp = np.ascontiguousarray(sub_ptr, dtype=np.int64)
    P = len(sp) - 1
    owner = np.zeros(P, dtype=np.int32)
    load = np.zeros(world, dtype=np.float64)
    check(load_library().gbe_shard_assign(P, _ptr(sp), int(world), _ptr(owner), _ptr(load)), "gbe_shard_assign")
    return owner, load


def parts_shard(ctx, parts, owner, rank):
    """The subgraphs of `parts` that `rank` owns, as a shard (gbe_parts_shard)."""
    ow = np.ascontiguousarray(owner, dtype=np.int32)
    h = ctypes.c_void_p()
    check(load_library().gbe_parts_shard(ctx.handle, parts.handle, _ptr(ow), int(rank), ctypes.byref(h)),
          "gbe_parts_shard")
    return Parts(ctx, h)


def dist_exchange(group=None):
    """Trace exchange of a sharded run over torch.distributed: an in-place all-reduce (sum)
    of the library's exchange buffer.  With NCCL the buffer is device memory and the
    all-reduce is ordered after the library's kernels on the current CUDA stream (the
    context must use that stream); with gloo (host ranks) the buffer is host memory."""
    import torch
    import torch.distributed as dist

    def fn(ptr, count, stream):
        if dist.get_backend(group) == "nccl":
            class _A:
                pass
            a = _A()
            a.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8", "data": (int(ptr), False),
                                          "version": 3}
            t = torch.as_tensor(a, device="cuda")
        else:
            t = torch.from_numpy(np.ctypeslib.as_array((ctypes.c_double * int(count)).from_address(int(ptr))))
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return fn


def subs_create(ctx, parts, prec):
    h = ctypes.c_void_p()
    check(load_library().gbe_subs_create(ctx.handle, parts.handle, prec, ctypes.byref(h)), "gbe_subs_create")
    return Subs(ctx, h)


def sp2_run(ctx, H, parts, params, X):
    check(load_library().gbe_sp2_run(ctx.handle, ctypes.byref(H), parts.handle, ctypes.byref(params), X.handle),
          "gbe_sp2_run")


def sp2_replay_batched(ctx, H, parts, params, budget_bytes, col, val, drop_tol=0.0):
    """Replayed SP2 in batches of subgraphs whose iterates fit budget_bytes, D into the
    caller's ELL buffers col[n, width], val[n, width]; returns the number of batches."""
    n, width = col.shape
    e = Ell(n, width, _ptr(col), _ptr(val), 1 if _is_device(col) else 0)
    b = ctypes.c_int()
    check(load_library().gbe_sp2_replay_batched(ctx.handle, ctypes.byref(H), parts.handle, ctypes.byref(params),
                                                int(budget_bytes), float(drop_tol), ctypes.byref(e), ctypes.byref(b)),
          "gbe_sp2_replay_batched")
    return b.value


def sp2_report_get(ctx, X):
    r = Sp2Report()
    check(load_library().gbe_sp2_report_get(ctx.handle, X.handle, ctypes.byref(r)), "gbe_sp2_report_get")
    return r


def subs_get_config(X):
    c = TcConfig()
    check(load_library().gbe_subs_get_config(X.handle, ctypes.byref(c)), "gbe_subs_get_config")
    return dict(stages=c.stages, schedule=c.schedule, kchunk=c.kchunk)


def subs_set_config(ctx, X, stages=0, schedule=SCHED_ROUND_ROBIN, kchunk=0):
    c = TcConfig(stages, schedule, kchunk)
    check(load_library().gbe_subs_set_config(ctx.handle, X.handle, ctypes.byref(c)), "gbe_subs_set_config")


def sp2_autotune(ctx, H, parts, params, X, reps=3):
    """Time every built squaring configuration on this problem, install the fastest; returns the report dict."""
    r = TuneReport()
    check(load_library().gbe_sp2_autotune(ctx.handle, ctypes.byref(H), parts.handle, ctypes.byref(params), X.handle,
                                          reps, ctypes.byref(r)), "gbe_sp2_autotune")
    return r.as_dict()


def sp2_submatrices(ctx, H, parts, params, X=None):
    """Returns (Subs, report dict).  Raises GbeError on failure (incl. ENOCONV)."""
    h = ctypes.c_void_p(X.handle.value if X is not None else None)
    r = Sp2Report()
    code = load_library().gbe_sp2_submatrices(ctx.handle, ctypes.byref(H), parts.handle, ctypes.byref(params),
                                              ctypes.byref(h), ctypes.byref(r))
    if X is None and h.value:
        X = Subs(ctx, h)
    check(code, "gbe_sp2_submatrices")
    return X, r.as_dict()


def sp2_gap_estimate(report, n_occ, e_lo=1e-6, e_hi=1e-2):
    """(homo, lumo) from a report dict (iters, eps, seq, t1, t2) of a finished run."""
    r = Sp2Report()
    r.iters = int(report["iters"])
    r.eps_min, r.eps_max = report["eps"]
    for i, b in enumerate(report["seq"]):
        r.seq[i] = int(b)
    for i, (a, b) in enumerate(zip(report["t1"], report["t2"])):
        r.t1[i], r.t2[i] = a, b
    homo, lumo = ctypes.c_double(), ctypes.c_double()
    check(load_library().gbe_sp2_gap_estimate(ctypes.byref(r), float(n_occ), float(e_lo), float(e_hi),
                                              ctypes.byref(homo), ctypes.byref(lumo)), "gbe_sp2_gap_estimate")
    return homo.value, lumo.value


def sp2_sequence(eps, homo, lumo, tol, n_max=SEQ_MAX):
    """Branch sequence (list of 0/1) that converges a gap [homo, lumo] within tol."""
    buf = (ctypes.c_uint8 * SEQ_MAX)()
    n = ctypes.c_int()
    check(load_library().gbe_sp2_sequence(float(eps[0]), float(eps[1]), float(homo), float(lumo), float(tol),
                                          int(n_max), ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(n)), "gbe_sp2_sequence")
    return list(buf[:n.value])


class FoeParams(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("mu", ctypes.c_double), ("order", ctypes.c_int),
                ("coeffs", ctypes.c_void_p), ("prec", ctypes.c_int), ("eps_given", ctypes.c_int),
                ("eps_min", ctypes.c_double), ("eps_max", ctypes.c_double), ("timeout_ms", ctypes.c_double)]


class FoeReport(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("status", ctypes.c_int), ("scale", ctypes.c_double),
                ("eps_min", ctypes.c_double), ("eps_max", ctypes.c_double), ("ms_gather", ctypes.c_float),
                ("ms_steps", ctypes.c_float), ("mma_flops", ctypes.c_double), ("alg_flops", ctypes.c_double)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


def fermi_coefficients(beta, mu, eps, order):
    c = np.zeros(order + 1)
    check(load_library().gbe_fermi_coefficients(float(beta), float(mu), float(eps[0]), float(eps[1]), int(order),
                                                _ptr(c)), "gbe_fermi_coefficients")
    return c


def foe_run(ctx, H, parts, X, beta, mu, order, prec=PREC_FP64, coeffs=None, eps=None, timeout_ms=0.0):
    """Enqueue a finite-temperature Chebyshev expansion into the state X; returns its report."""
    cbuf = None if coeffs is None else np.ascontiguousarray(coeffs, dtype=np.float64)
    p = FoeParams(float(beta), float(mu), int(order), _ptr(cbuf) if cbuf is not None else None, int(prec),
                  1 if eps is not None else 0, eps[0] if eps is not None else 0.0,
                  eps[1] if eps is not None else 0.0, float(timeout_ms))
    check(load_library().gbe_foe_run(ctx.handle, ctypes.byref(H), parts.handle, ctypes.byref(p), X.handle),
          "gbe_foe_run")
    r = FoeReport()
    check(load_library().gbe_foe_report_get(ctx.handle, X.handle, ctypes.byref(r)), "gbe_foe_report_get")
    return r.as_dict()


def gershgorin_noalloc(ctx, H, bounds):
    """Enqueue allocation-free Gershgorin bounds of device CSR H into bounds (device, 2 doubles)."""
    check(load_library().gbe_gershgorin_noalloc(ctx.handle, ctypes.byref(H), _ptr(bounds)),
          "gbe_gershgorin_noalloc")
    return bounds


def assemble_width(ctx, X, parts):
    e = Ell()
    check(load_library().gbe_assemble_D(ctx.handle, X.handle, parts.handle, 0.0, ctypes.byref(e)), "gbe_assemble_D")
    return e.n, e.width


def assemble_D(ctx, X, parts, col, val, drop_tol=0.0):
    """Fill caller-owned ELL buffers col[n, width] (int32) and val[n, width] (float64)."""
    n, width = col.shape
    e = Ell(n, width, _ptr(col), _ptr(val), 1 if _is_device(col) else 0)
    check(load_library().gbe_assemble_D(ctx.handle, X.handle, parts.handle, float(drop_tol), ctypes.byref(e)),
          "gbe_assemble_D")
    return col, val


def ell_struct(col, val):
    n, width = col.shape
    e = Ell(n, width, _ptr(col), _ptr(val), 1 if _is_device(col) else 0)
    e._keep = (col, val)
    return e


def ell_to_dense(col, val, n):
    """Dense D from an ELL pair (row i of the ELL = column i of D).  Test/inspection helper."""
    col = np.asarray(col)
    val = np.asarray(val)
    D = np.zeros((n, n))
    rows = np.repeat(np.arange(n), col.shape[1]).reshape(col.shape)
    m = col >= 0
    D[col[m], rows[m]] = val[m]
    return D


# ----------------------------------------------------------------------------- learned graph proposal
class Pairs(_Owned):
    _free = "gbe_free_pairs"

    def info(self):
        n, npairs = ctypes.c_int64(), ctypes.c_int64()
        check(load_library().gbe_pairs_info(self._h, ctypes.byref(n), ctypes.byref(npairs)), "gbe_pairs_info")
        return n.value, npairs.value

    def export(self):
        """(rowptr[n+1], j[npairs], features[npairs, 5]) as NumPy arrays."""
        n, npairs = self.info()
        rp = np.zeros(n + 1, dtype=np.int64)
        j = np.zeros(max(npairs, 1), dtype=np.int32)
        f = np.zeros((max(npairs, 1), 5), dtype=np.float32)
        check(load_library().gbe_pairs_export(self.ctx.handle, self._h, _ptr(rp), _ptr(j), _ptr(f)), "gbe_pairs_export")
        return rp, j[:npairs], f[:npairs]

    def device(self):
        """(rowptr, j, features) device addresses (library-owned, valid while this object lives)."""
        rp, j, f = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        check(load_library().gbe_pairs_device(self._h, ctypes.byref(rp), ctypes.byref(j), ctypes.byref(f)),
              "gbe_pairs_device")
        return rp.value, j.value, f.value


class Mlp(_Owned):
    _free = "gbe_free_mlp"

    @property
    def param_count(self):
        return load_library().gbe_mlp_param_count(self._h)

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.param_count
        check(load_library().gbe_mlp_set_params(self.ctx.handle, self._h, _ptr(p)), "gbe_mlp_set_params")

    def get_params(self):
        p = np.zeros(self.param_count, dtype=np.float32)
        check(load_library().gbe_mlp_get_params(self.ctx.handle, self._h, _ptr(p)), "gbe_mlp_get_params")
        return p

    def forward(self, pairs, logits):
        check(load_library().gbe_mlp_forward(self.ctx.handle, self._h, pairs.handle, _ptr(logits)), "gbe_mlp_forward")
        return logits

    def gradient(self, pairs, labels):
        loss = ctypes.c_double()
        g = np.zeros(self.param_count, dtype=np.float32)
        check(load_library().gbe_mlp_gradient(self.ctx.handle, self._h, pairs.handle, _ptr(labels), ctypes.byref(loss),
                                              _ptr(g)), "gbe_mlp_gradient")
        return loss.value, g

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        check(load_library().gbe_mlp_adam_step(self.ctx.handle, self._h, lr, beta1, beta2, eps), "gbe_mlp_adam_step")

    def train(self, pairs, labels, epochs, lr):
        loss = ctypes.c_double()
        check(load_library().gbe_mlp_train(self.ctx.handle, self._h, pairs.handle, _ptr(labels), int(epochs),
                                           float(lr), ctypes.byref(loss)), "gbe_mlp_train")
        return loss.value


def pairs_build(ctx, site_struct, H, rcand):
    h = ctypes.c_void_p()
    check(load_library().gbe_pairs_build(ctx.handle, ctypes.byref(site_struct), ctypes.byref(H), float(rcand),
                                         ctypes.byref(h)), "gbe_pairs_build")
    return Pairs(ctx, h)


def mlp_labels(ctx, pairs, col, val, tau, labels):
    """Enqueue the training labels of the pairs (device uint8[npairs]) from a device ELL D."""
    e = ell_struct(col, val)
    check(load_library().gbe_mlp_labels(ctx.handle, pairs.handle, ctypes.byref(e), float(tau), _ptr(labels)),
          "gbe_mlp_labels")
    return labels


def mlp_create(ctx, hidden=64):
    h = ctypes.c_void_p()
    check(load_library().gbe_mlp_create(ctx.handle, int(hidden), ctypes.byref(h)), "gbe_mlp_create")
    return Mlp(ctx, h)
