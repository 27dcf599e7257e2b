"""Thin ctypes binding of librosen.so (include/rosen.h).

Every function here only marshals arguments: PyTorch tensors are passed as
raw device pointers, PyTorch streams as their cudaStream_t handle, and the
work runs in the library's CUDA kernels.  There is no fallback: if the
library is missing or was built without a GPU to run on, calls raise.
"""
import ctypes
import os

import torch

from . import build as _build

# ---- constants mirrored from rosen.h -------------------------------------
ROSEN_OK, ROSEN_EINVAL, ROSEN_ENOMEM, ROSEN_ECUDA = 0, 1, 2, 3
ROSEN_ETIMEOUT, ROSEN_EBUSY, ROSEN_EAGAIN, ROSEN_ECLOSED, ROSEN_ENOTFOUND = 4, 5, 6, 7, 8
ROSEN_LATTICE_NMAX = 512
ROSEN_LATTICE_LONG_NMAX = 32768
ROSEN_MAX_ATTEMPTS = 65535
ROSEN_OFFLATTICE_NMAX = 1024
ROSEN_OFFLATTICE_LONG_NMAX = 16384
ROSEN_KMAX = 128
ROSEN_STORE_TRACE = 1
ROSEN_STORE_COORDS = 2
ROSEN_HARD_SPHERE = 0
ROSEN_LJ = 1
ROSEN_REDUCE_LATTICE = 0
ROSEN_REDUCE_OFFLATTICE = 1

STAT_KEYS = ["n", "n_alive", "log_max", "S0", "S1", "S2", "Q0", "Q1_r2", "Q2_r2",
             "Q1_rg2", "Q2_rg2", "logZ", "logZ_norm", "mean_r2", "se_r2", "mean_rg2",
             "se_rg2", "ess"]


class RosenError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (status_string(status), message))
        self.status = status


_vp = ctypes.c_void_p


class rosen_lattice_params(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("ensemble", ctypes.c_uint32),
                ("N", ctypes.c_int32), ("C", ctypes.c_int64), ("chain0", ctypes.c_int64),
                ("beta_eps", ctypes.c_double), ("flags", ctypes.c_uint32),
                ("lanes_per_chain", ctypes.c_int32), ("max_attempts", ctypes.c_int32)]


class rosen_lattice_out(ctypes.Structure):
    _fields_ = [("counts", _vp), ("logw", _vp), ("r2", _vp), ("n2rg2", _vp),
                ("trace", _vp), ("coords", _vp), ("attempts", _vp)]


class rosen_offlattice_params(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("ensemble", ctypes.c_uint32),
                ("N", ctypes.c_int32), ("C", ctypes.c_int64), ("chain0", ctypes.c_int64),
                ("k", ctypes.c_int32), ("potential", ctypes.c_int32), ("sigma", ctypes.c_double),
                ("cutoff", ctypes.c_double), ("beta_eps", ctypes.c_double),
                ("flags", ctypes.c_uint32), ("lanes_per_chain", ctypes.c_int32),
                ("max_attempts", ctypes.c_int32)]


class rosen_offlattice_out(ctypes.Structure):
    _fields_ = [("logw", _vp), ("r2", _vp), ("rg2", _vp), ("alive", _vp), ("trace", _vp),
                ("coords", _vp), ("counters", _vp), ("attempts", _vp)]


class rosen_reduce_in(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("N", ctypes.c_int32), ("k", ctypes.c_int32),
                ("use_counts", ctypes.c_int32), ("C", ctypes.c_int64), ("logw", _vp),
                ("counts", _vp), ("r2_i", _vp), ("n2rg2", _vp), ("r2_f", _vp),
                ("rg2_f", _vp), ("attempts", _vp)]


ROSEN_MODEL_LATTICE = 0
ROSEN_MODEL_OFFLATTICE = 1
ROSEN_PERM_MAX_POP = 1 << 24


class rosen_perm_params(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("ensemble", ctypes.c_uint32), ("N", ctypes.c_int32),
                ("M0", ctypes.c_int64), ("max_population", ctypes.c_int64),
                ("beta_eps", ctypes.c_double), ("mu", ctypes.c_double), ("c_hi", ctypes.c_double),
                ("c_lo", ctypes.c_double), ("flags", ctypes.c_uint32), ("reserved", ctypes.c_int32)]


class rosen_perm_out(ctypes.Structure):
    _fields_ = [("population", _vp), ("logz", _vp), ("mean_r2", _vp), ("final_n", _vp),
                ("w_m", _vp), ("w_e", _vp), ("coords", _vp)]


class rosen_ensemble(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("N", ctypes.c_int32), ("C", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("ensemble", ctypes.c_uint32), ("k", ctypes.c_int32),
                ("potential", ctypes.c_int32), ("max_attempts", ctypes.c_int32),
                ("beta_eps", ctypes.c_double), ("sigma", ctypes.c_double),
                ("cutoff", ctypes.c_double)]


_LIB = None


def library_path():
    return _build.LIB


def load():
    """Load librosen.so; raise if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError("librosen.so is not built (%s); run paper_1704_04381_gb300.build.build()"
                           % path)
    L = ctypes.CDLL(path)
    L.rosen_status_string.argtypes = [ctypes.c_int]
    L.rosen_status_string.restype = ctypes.c_char_p
    L.rosen_last_error.argtypes = []
    L.rosen_last_error.restype = ctypes.c_char_p
    L.rosen_version.argtypes = []
    L.rosen_version.restype = ctypes.c_char_p
    L.rosen_philox.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                               ctypes.c_int64, ctypes.c_int64, _vp, _vp]
    L.rosen_philox.restype = ctypes.c_int
    L.rosen_lattice_grow.argtypes = [ctypes.POINTER(rosen_lattice_params),
                                     ctypes.POINTER(rosen_lattice_out), _vp]
    L.rosen_lattice_grow.restype = ctypes.c_int
    L.rosen_lattice_long_workspace_size.argtypes = [ctypes.c_int32, ctypes.c_int64]
    L.rosen_lattice_long_workspace_size.restype = ctypes.c_size_t
    L.rosen_lattice_grow_long.argtypes = [ctypes.POINTER(rosen_lattice_params),
                                          ctypes.POINTER(rosen_lattice_out), _vp, ctypes.c_size_t,
                                          _vp]
    L.rosen_lattice_grow_long.restype = ctypes.c_int
    L.rosen_offlattice_long_workspace_size.argtypes = [ctypes.c_int32, ctypes.c_int64]
    L.rosen_offlattice_long_workspace_size.restype = ctypes.c_size_t
    L.rosen_offlattice_grow_long.argtypes = [ctypes.POINTER(rosen_offlattice_params),
                                             ctypes.POINTER(rosen_offlattice_out), _vp,
                                             ctypes.c_size_t, _vp]
    L.rosen_offlattice_grow_long.restype = ctypes.c_int
    L.rosen_offlattice_grow.argtypes = [ctypes.POINTER(rosen_offlattice_params),
                                        ctypes.POINTER(rosen_offlattice_out), _vp]
    L.rosen_offlattice_grow.restype = ctypes.c_int
    L.rosen_sphere_points.argtypes = [_vp, ctypes.c_int64, _vp, _vp]
    L.rosen_sphere_points.restype = ctypes.c_int
    L.rosen_sphere_points_ff.argtypes = [_vp, ctypes.c_int64, _vp, _vp]
    L.rosen_sphere_points_ff.restype = ctypes.c_int
    L.rosen_reduce_workspace_size.argtypes = [ctypes.c_int64]
    L.rosen_reduce_workspace_size.restype = ctypes.c_size_t
    L.rosen_reduce.argtypes = [ctypes.POINTER(rosen_reduce_in), _vp, _vp, ctypes.c_size_t, _vp]
    L.rosen_reduce.restype = ctypes.c_int
    L.rosen_batch_create.argtypes = [ctypes.POINTER(rosen_ensemble), ctypes.c_int32,
                                     ctypes.POINTER(_vp)]
    L.rosen_batch_create.restype = ctypes.c_int
    for name in ("rosen_batch_tune", "rosen_batch_run"):
        getattr(L, name).argtypes = [_vp, _vp]
        getattr(L, name).restype = ctypes.c_int
    L.rosen_batch_copy_stats.argtypes = [_vp, _vp, _vp]
    L.rosen_batch_copy_stats.restype = ctypes.c_int
    L.rosen_batch_copy_lattice.argtypes = [_vp, ctypes.c_int32, ctypes.POINTER(rosen_lattice_out),
                                           _vp]
    L.rosen_batch_copy_lattice.restype = ctypes.c_int
    L.rosen_batch_copy_offlattice.argtypes = [_vp, ctypes.c_int32,
                                              ctypes.POINTER(rosen_offlattice_out), _vp]
    L.rosen_batch_copy_offlattice.restype = ctypes.c_int
    L.rosen_batch_counters.argtypes = [_vp, _vp, _vp]
    L.rosen_batch_counters.restype = ctypes.c_int
    L.rosen_batch_describe.argtypes = [_vp, ctypes.c_char_p, ctypes.c_size_t]
    L.rosen_batch_describe.restype = ctypes.c_int
    L.rosen_batch_destroy.argtypes = [_vp]
    L.rosen_batch_destroy.restype = ctypes.c_int
    L.rosen_reduce_noalloc.argtypes = [ctypes.POINTER(rosen_reduce_in), _vp, _vp]
    L.rosen_reduce_noalloc.restype = ctypes.c_int
    L.rosen_stats_merge.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp]
    L.rosen_stats_merge.restype = ctypes.c_int
    L.rosen_perm_workspace_size.argtypes = [ctypes.c_int32, ctypes.c_int64]
    L.rosen_perm_workspace_size.restype = ctypes.c_size_t
    L.rosen_perm_run.argtypes = [ctypes.POINTER(rosen_perm_params), ctypes.POINTER(rosen_perm_out),
                                 _vp, ctypes.c_size_t, _vp]
    L.rosen_perm_run.restype = ctypes.c_int
    _LIB = L
    return L


def status_string(status):
    return load().rosen_status_string(int(status)).decode()


def last_error():
    return load().rosen_last_error().decode()


def version():
    return load().rosen_version().decode()


def _check(status):
    if status != ROSEN_OK:
        raise RosenError(status, last_error())


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError("librosen takes device tensors")
    if not t.is_contiguous():
        raise ValueError("librosen takes contiguous tensors")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


# ---- entry points ----------------------------------------------------------
def rosen_philox(seed, ensemble, step, slot, chain0, n, out, stream=None):
    """out [n, 4] uint32 (int32 tensor) <- Philox4x32-10 of counters (chain0+q, ensemble, step, slot)."""
    _check(load().rosen_philox(int(seed), int(ensemble), int(step), int(slot), int(chain0),
                               int(n), _ptr(out), _stream(stream)))


def rosen_lattice_grow(params, out, stream=None):
    """Grow lattice chains.  params: rosen_lattice_params; out: dict of tensors."""
    o = rosen_lattice_out(counts=_ptr(out.get("counts")), logw=_ptr(out.get("logw")),
                          r2=_ptr(out.get("r2")), n2rg2=_ptr(out.get("n2rg2")),
                          trace=_ptr(out.get("trace")), coords=_ptr(out.get("coords")),
                          attempts=_ptr(out.get("attempts")))
    _check(load().rosen_lattice_grow(ctypes.byref(params), ctypes.byref(o), _stream(stream)))


def rosen_lattice_long_workspace_size(N, C):
    return int(load().rosen_lattice_long_workspace_size(int(N), int(C)))


def lattice_long_workspace(N, C, device="cuda"):
    """Allocate the hash-table workspace of rosen_lattice_grow_long."""
    nbytes = rosen_lattice_long_workspace_size(N, C)
    return torch.empty(max(nbytes, 8) // 8, dtype=torch.int64, device=device)


def rosen_lattice_grow_long(params, out, workspace, stream=None):
    """Grow long lattice chains (N <= 32768) with per-chain hash tables in workspace."""
    o = rosen_lattice_out(counts=_ptr(out.get("counts")), logw=_ptr(out.get("logw")),
                          r2=_ptr(out.get("r2")), n2rg2=_ptr(out.get("n2rg2")),
                          trace=_ptr(out.get("trace")), coords=_ptr(out.get("coords")),
                          attempts=_ptr(out.get("attempts")))
    _check(load().rosen_lattice_grow_long(ctypes.byref(params), ctypes.byref(o), _ptr(workspace),
                                          workspace.numel() * workspace.element_size(),
                                          _stream(stream)))


def rosen_offlattice_grow(params, out, stream=None):
    """Grow real-space chains.  params: rosen_offlattice_params; out: dict of tensors."""
    o = rosen_offlattice_out(logw=_ptr(out.get("logw")), r2=_ptr(out.get("r2")),
                             rg2=_ptr(out.get("rg2")), alive=_ptr(out.get("alive")),
                             trace=_ptr(out.get("trace")), coords=_ptr(out.get("coords")),
                             counters=_ptr(out.get("counters")),
                             attempts=_ptr(out.get("attempts")))
    _check(load().rosen_offlattice_grow(ctypes.byref(params), ctypes.byref(o), _stream(stream)))


def rosen_sphere_points_ff(words, out, stream=None):
    """out [n, 5] float32 <- float-float directions (x hi, x lo, y hi, y lo, z) of words [n, 2]."""
    n = words.shape[0]
    _check(load().rosen_sphere_points_ff(_ptr(words), int(n), _ptr(out), _stream(stream)))


def rosen_offlattice_long_workspace_size(N, C):
    return int(load().rosen_offlattice_long_workspace_size(int(N), int(C)))


def offlattice_long_workspace(N, C, device="cuda"):
    """Allocate the per-chain-slot workspace of rosen_offlattice_grow_long."""
    nbytes = rosen_offlattice_long_workspace_size(N, C)
    return torch.empty(max(nbytes, 16) // 16 * 2, dtype=torch.int64, device=device)


def rosen_offlattice_grow_long(params, out, workspace, stream=None):
    """Grow long real-space chains (N <= 16384) with cell grids in workspace."""
    o = rosen_offlattice_out(logw=_ptr(out.get("logw")), r2=_ptr(out.get("r2")),
                             rg2=_ptr(out.get("rg2")), alive=_ptr(out.get("alive")),
                             trace=_ptr(out.get("trace")), coords=_ptr(out.get("coords")),
                             counters=_ptr(out.get("counters")),
                             attempts=_ptr(out.get("attempts")))
    _check(load().rosen_offlattice_grow_long(ctypes.byref(params), ctypes.byref(o),
                                             _ptr(workspace),
                                             workspace.numel() * workspace.element_size(),
                                             _stream(stream)))


def rosen_sphere_points(words, out, stream=None):
    """out [n, 3] float32 <- the kernels' trial directions of word pairs words [n, 2]."""
    n = words.shape[0]
    _check(load().rosen_sphere_points(_ptr(words), int(n), _ptr(out), _stream(stream)))


def rosen_reduce_workspace_size(C):
    return int(load().rosen_reduce_workspace_size(int(C)))


def rosen_reduce(inp, stats, workspace, stream=None):
    """Reduce per-chain outputs (rosen_reduce_in built from tensors) into stats [18] float64."""
    _check(load().rosen_reduce(ctypes.byref(inp), _ptr(stats), _ptr(workspace),
                               workspace.numel() * workspace.element_size(), _stream(stream)))


ROSEN_REDUCE_NOALLOC_MAX_CHAINS = 1 << 24


def rosen_reduce_noalloc(inp, stats, stream=None):
    """rosen_reduce with the library's built-in scratch: for callers that cannot
    allocate device memory (C <= 2^24; calls that overlap on the GPU race)."""
    _check(load().rosen_reduce_noalloc(ctypes.byref(inp), _ptr(stats), _stream(stream)))


# ---- conveniences (allocation only) ---------------------------------------
def lattice_params(seed, N, C, beta_eps=0.0, ensemble=0, chain0=0, flags=0, lanes_per_chain=0,
                   max_attempts=0):
    return rosen_lattice_params(seed=int(seed), ensemble=int(ensemble), N=int(N), C=int(C),
                                chain0=int(chain0), beta_eps=float(beta_eps), flags=int(flags),
                                lanes_per_chain=int(lanes_per_chain),
                                max_attempts=int(max_attempts))


def lattice_outputs(N, C, device="cuda", trace=False, coords=False, attempts=False):
    """Allocate the per-chain output tensors of rosen_lattice_grow."""
    out = {
        "counts": torch.empty((C, 8), dtype=torch.int16, device=device),
        "logw": torch.empty(C, dtype=torch.float32, device=device),
        "r2": torch.empty(C, dtype=torch.int32, device=device),
        "n2rg2": torch.empty(C, dtype=torch.int64, device=device),
    }
    if attempts:
        out["attempts"] = torch.empty(C, dtype=torch.int16, device=device)
    if trace:
        out["trace"] = torch.empty((N - 1, C), dtype=torch.uint8, device=device)
    if coords:
        out["coords"] = torch.empty((N, 3, C), dtype=torch.int32, device=device)
    return out


def offlattice_params(seed, N, C, k, potential=ROSEN_HARD_SPHERE, beta_eps=0.0, sigma=1.0,
                      cutoff=2.5, ensemble=0, chain0=0, flags=0, lanes_per_chain=0,
                      max_attempts=0):
    return rosen_offlattice_params(seed=int(seed), ensemble=int(ensemble), N=int(N), C=int(C),
                                   chain0=int(chain0), k=int(k), potential=int(potential),
                                   sigma=float(sigma), cutoff=float(cutoff),
                                   beta_eps=float(beta_eps), flags=int(flags),
                                   lanes_per_chain=int(lanes_per_chain),
                                   max_attempts=int(max_attempts))


def offlattice_outputs(N, C, device="cuda", trace=False, coords=False, counters=False,
                       attempts=False):
    """Allocate the per-chain output tensors of rosen_offlattice_grow."""
    out = {
        "logw": torch.empty(C, dtype=torch.float32, device=device),
        "r2": torch.empty(C, dtype=torch.float32, device=device),
        "rg2": torch.empty(C, dtype=torch.float32, device=device),
        "alive": torch.empty(C, dtype=torch.uint8, device=device),
    }
    if attempts:
        out["attempts"] = torch.empty(C, dtype=torch.int16, device=device)
    if trace:
        out["trace"] = torch.empty((N - 1, C), dtype=torch.uint8, device=device)
    if coords:
        out["coords"] = torch.empty((N, 3, C), dtype=torch.float32, device=device)
    if counters:
        out["counters"] = torch.zeros(3, dtype=torch.int64, device=device)
    return out


def offlattice_reduce_in(out, N, k):
    """Reduction inputs of real-space outputs (with their attempts, if any)."""
    C = out["logw"].numel()
    return rosen_reduce_in(kind=ROSEN_REDUCE_OFFLATTICE, N=int(N), k=int(k), use_counts=0, C=C,
                           logw=_ptr(out["logw"]), counts=None, r2_i=None, n2rg2=None,
                           r2_f=_ptr(out["r2"]), rg2_f=_ptr(out["rg2"]),
                           attempts=_ptr(out.get("attempts")))


def lattice_reduce_in(out, N, use_counts):
    """Reduction inputs of lattice outputs (with their attempts, if any)."""
    C = out["logw"].numel()
    return rosen_reduce_in(kind=ROSEN_REDUCE_LATTICE, N=int(N), k=0, use_counts=int(use_counts),
                           C=C, logw=_ptr(out["logw"]), counts=_ptr(out["counts"]),
                           r2_i=_ptr(out["r2"]), n2rg2=_ptr(out["n2rg2"]), r2_f=None, rg2_f=None,
                           attempts=_ptr(out.get("attempts")))


def rosen_stats_merge(parts, N, k=0):
    """Merge rosen_stats of disjoint chain sets (host sequences of 18 numbers
    in STAT_KEYS order, or dicts) into the statistics of their union; runs
    in the library, on the host."""
    rows = [[p[key] for key in STAT_KEYS] if isinstance(p, dict) else list(p) for p in parts]
    n = len(rows)
    arr = (ctypes.c_double * (len(STAT_KEYS) * max(n, 1)))(*[v for r in rows for v in r])
    out = (ctypes.c_double * len(STAT_KEYS))()
    _check(load().rosen_stats_merge(ctypes.cast(arr, _vp), int(n), int(N), int(k),
                                    ctypes.cast(out, _vp)))
    return dict(zip(STAT_KEYS, list(out)))


def perm_params(seed, N, M0, max_population=None, beta_eps=0.0, mu=4.684, c_hi=3.0,
                c_lo=1.0 / 3.0, ensemble=0, flags=0):
    return rosen_perm_params(seed=int(seed), ensemble=int(ensemble), N=int(N), M0=int(M0),
                             max_population=int(max_population or 4 * M0),
                             beta_eps=float(beta_eps), mu=float(mu), c_hi=float(c_hi),
                             c_lo=float(c_lo), flags=int(flags), reserved=0)


def perm_outputs(N, max_population, device="cuda", coords=False):
    """Allocate the outputs of rosen_perm_run (final weights always)."""
    out = {
        "population": torch.empty(N, dtype=torch.int64, device=device),
        "logz": torch.empty(N, dtype=torch.float64, device=device),
        "mean_r2": torch.empty(N, dtype=torch.float64, device=device),
        "final_n": torch.empty(1, dtype=torch.int64, device=device),
        "w_m": torch.empty(max_population, dtype=torch.float64, device=device),
        "w_e": torch.empty(max_population, dtype=torch.int32, device=device),
    }
    if coords:
        out["coords"] = torch.empty((N, 3, max_population), dtype=torch.int32, device=device)
    return out


def perm_workspace(N, max_population, device="cuda"):
    nbytes = int(load().rosen_perm_workspace_size(int(N), int(max_population)))
    if nbytes == 0:
        raise RosenError(ROSEN_EINVAL, "PERM sizes out of range")
    return torch.empty((nbytes + 255) // 256 * 32, dtype=torch.float64, device=device)


def rosen_perm_run(params, out, workspace, stream=None):
    """PERM on the cubic lattice (breadth first); out from perm_outputs."""
    o = rosen_perm_out(population=_ptr(out["population"]), logz=_ptr(out["logz"]),
                       mean_r2=_ptr(out.get("mean_r2")), final_n=_ptr(out["final_n"]),
                       w_m=_ptr(out.get("w_m")), w_e=_ptr(out.get("w_e")),
                       coords=_ptr(out.get("coords")))
    _check(load().rosen_perm_run(ctypes.byref(params), ctypes.byref(o), _ptr(workspace),
                                 workspace.numel() * workspace.element_size(), _stream(stream)))


def stats_tensor(device="cuda"):
    return torch.empty(len(STAT_KEYS), dtype=torch.float64, device=device)


def stats_dict(t):
    return dict(zip(STAT_KEYS, t.detach().cpu().tolist()))


def reduce_workspace(C, device="cuda"):
    nbytes = rosen_reduce_workspace_size(C)
    return torch.empty((nbytes + 15) // 16 * 2, dtype=torch.float64, device=device)


# ---- batched growth ----------------------------------------------------------
def ensemble(model, N, C, seed, ensemble_id=0, k=0, potential=ROSEN_HARD_SPHERE, beta_eps=0.0,
             sigma=1.0, cutoff=2.5, max_attempts=0):
    return rosen_ensemble(model=int(model), N=int(N), C=int(C), seed=int(seed),
                          ensemble=int(ensemble_id), k=int(k), potential=int(potential),
                          max_attempts=int(max_attempts), beta_eps=float(beta_eps),
                          sigma=float(sigma), cutoff=float(cutoff))


class RosenBatch:
    """A planned batch of ensembles (rosen_batch_*): tune, run, read back."""

    def __init__(self, ensembles):
        arr = (rosen_ensemble * len(ensembles))(*ensembles)
        self.ensembles = list(ensembles)
        h = _vp()
        _check(load().rosen_batch_create(arr, len(ensembles), ctypes.byref(h)))
        self.handle = h

    def tune(self, stream=None):
        _check(load().rosen_batch_tune(self.handle, _stream(stream)))

    def run(self, stream=None):
        _check(load().rosen_batch_run(self.handle, _stream(stream)))

    def stats(self, out=None, stream=None):
        if out is None:
            out = torch.empty((len(self.ensembles), len(STAT_KEYS)), dtype=torch.float64,
                              device="cuda")
        _check(load().rosen_batch_copy_stats(self.handle, _ptr(out), _stream(stream)))
        return out

    def lattice_outputs(self, e, stream=None):
        ens = self.ensembles[e]
        out = lattice_outputs(ens.N, ens.C, attempts=ens.max_attempts > 1)
        o = rosen_lattice_out(counts=_ptr(out["counts"]), logw=_ptr(out["logw"]),
                              r2=_ptr(out["r2"]), n2rg2=_ptr(out["n2rg2"]),
                              attempts=_ptr(out.get("attempts")))
        _check(load().rosen_batch_copy_lattice(self.handle, int(e), ctypes.byref(o), _stream(stream)))
        return out

    def offlattice_outputs(self, e, stream=None):
        ens = self.ensembles[e]
        out = offlattice_outputs(ens.N, ens.C, attempts=ens.max_attempts > 1)
        o = rosen_offlattice_out(logw=_ptr(out["logw"]), r2=_ptr(out["r2"]),
                                 rg2=_ptr(out["rg2"]), alive=_ptr(out["alive"]),
                                 attempts=_ptr(out.get("attempts")))
        _check(load().rosen_batch_copy_offlattice(self.handle, int(e), ctypes.byref(o),
                                                  _stream(stream)))
        return out

    def counters(self, stream=None):
        out = torch.zeros(3, dtype=torch.int64, device="cuda")
        _check(load().rosen_batch_counters(self.handle, _ptr(out), _stream(stream)))
        return out

    def describe(self):
        buf = ctypes.create_string_buffer(1 << 16)
        _check(load().rosen_batch_describe(self.handle, buf, len(buf)))
        return buf.value.decode()

    def close(self):
        if self.handle:
            load().rosen_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- serving -----------------------------------------------------------------
class rosen_stats_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in STAT_KEYS]


class rosen_serve_config(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("max_slots", ctypes.c_int32),
                ("max_queue", ctypes.c_int32), ("device", ctypes.c_int32),
                ("shortest_first", ctypes.c_int32), ("pool_max_bytes", ctypes.c_uint64)]


class rosen_request(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("N", ctypes.c_int32), ("C", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("ensemble", ctypes.c_uint32), ("k", ctypes.c_int32),
                ("potential", ctypes.c_int32), ("store_coords", ctypes.c_int32),
                ("beta_eps", ctypes.c_double), ("sigma", ctypes.c_double),
                ("cutoff", ctypes.c_double), ("max_attempts", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class rosen_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("stats", rosen_stats_t),
                ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64), ("coords", _vp), ("message", ctypes.c_char * 256)]


class rosen_serve_counters(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "rejected", "completed", "failed",
                                               "queued", "running", "bytes_in_use")]


_SERVE_SIGS = {
    "rosen_serve_create": [ctypes.POINTER(rosen_serve_config), ctypes.POINTER(_vp)],
    "rosen_serve_submit": [_vp, ctypes.POINTER(rosen_request), ctypes.POINTER(ctypes.c_uint64)],
    "rosen_serve_poll": [_vp, ctypes.c_uint64, ctypes.POINTER(rosen_result)],
    "rosen_serve_wait": [_vp, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(rosen_result)],
    "rosen_serve_cancel": [_vp, ctypes.c_uint64],
    "rosen_serve_release": [_vp, ctypes.c_uint64],
    "rosen_serve_info": [_vp, ctypes.POINTER(rosen_serve_counters)],
    "rosen_serve_destroy": [_vp],
}


def _serve_lib():
    L = load()
    for name, args in _SERVE_SIGS.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    return L


def request(model, N, C, seed, ensemble_id=0, k=0, potential=ROSEN_HARD_SPHERE, beta_eps=0.0,
            sigma=1.0, cutoff=2.5, store_coords=False, max_attempts=0):
    return rosen_request(model=int(model), N=int(N), C=int(C), seed=int(seed),
                         ensemble=int(ensemble_id), k=int(k), potential=int(potential),
                         store_coords=int(bool(store_coords)), beta_eps=float(beta_eps),
                         sigma=float(sigma), cutoff=float(cutoff),
                         max_attempts=int(max_attempts), reserved=0)


def result_dict(r):
    return {"ticket": r.ticket, "status": r.status,
            "stats": {k: getattr(r.stats, k) for k in STAT_KEYS},
            "t_submit_ns": r.t_submit_ns, "t_admit_ns": r.t_admit_ns, "t_done_ns": r.t_done_ns,
            "coords": r.coords, "message": r.message.decode(errors="replace")}


class _DeviceArray:
    """A typed view of device memory the library owns (CUDA array interface)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(int(v) for v in shape),
                                         "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def served_coords(result, model, N, C):
    """Zero-copy torch view [N, 3, C] of a served request's stored
    conformations (int32 on the lattice, float32 in real space).  The memory
    belongs to the server and is valid until the ticket is released."""
    ptr = result["coords"]
    if not ptr:
        raise ValueError("the request stored no conformations")
    typestr = "<i4" if int(model) == ROSEN_MODEL_LATTICE else "<f4"
    return torch.as_tensor(_DeviceArray(ptr, (N, 3, C), typestr), device="cuda")


class RosenServer:
    """The request loop (rosen_serve_*): submit, poll/wait, release."""

    def __init__(self, mem_budget_bytes, max_slots=32, max_queue=4096, device=0,
                 shortest_first=False, pool_max_bytes=0):
        cfg = rosen_serve_config(mem_budget_bytes=int(mem_budget_bytes), max_slots=int(max_slots),
                                 max_queue=int(max_queue), device=int(device),
                                 shortest_first=int(bool(shortest_first)),
                                 pool_max_bytes=int(pool_max_bytes))
        h = _vp()
        _check(_serve_lib().rosen_serve_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h

    def submit(self, req):
        """Return the ticket, or raise RosenError (EBUSY, EINVAL, ECLOSED)."""
        t = ctypes.c_uint64()
        _check(_serve_lib().rosen_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def try_submit(self, req):
        """(status, ticket) without raising."""
        t = ctypes.c_uint64()
        st = _serve_lib().rosen_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(t))
        return st, t.value

    def poll(self, ticket):
        r = rosen_result()
        st = _serve_lib().rosen_serve_poll(self.handle, int(ticket), ctypes.byref(r))
        return st, (result_dict(r) if st == ROSEN_OK else None)

    def wait(self, ticket, timeout_s=60.0):
        r = rosen_result()
        st = _serve_lib().rosen_serve_wait(self.handle, int(ticket), int(timeout_s * 1e9),
                                           ctypes.byref(r))
        return st, (result_dict(r) if st == ROSEN_OK else None)

    def cancel(self, ticket):
        return _serve_lib().rosen_serve_cancel(self.handle, int(ticket))

    def release(self, ticket):
        return _serve_lib().rosen_serve_release(self.handle, int(ticket))

    def info(self):
        c = rosen_serve_counters()
        _check(_serve_lib().rosen_serve_info(self.handle, ctypes.byref(c)))
        return {k: getattr(c, k) for k, _ in c._fields_}

    def close(self):
        if self.handle:
            _serve_lib().rosen_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
