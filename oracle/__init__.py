"""Python face of the CPU oracle (test infrastructure only).

The oracle is a plain FP64 C implementation of Rosenbluth chain growth
(Guo & Baulin, arxiv 1704.04381: Eq. 3, Algorithms 1-2, Eq. 2 and Eq. 9) that
shares no code with the CUDA library.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` import this package; the product path never does.
"""
import ctypes
import os

import numpy as np

from . import build as _build

HARD_SPHERE = 0
LJ = 1

_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        f64p = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u16p = ctypes.POINTER(ctypes.c_uint16)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_philox4x32_10.restype = None
        L.orc_lattice_chain.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_int, ctypes.c_double, i32p, u8p, u16p,
                                        f64p, i64p, i64p]
        L.orc_lattice_chain.restype = ctypes.c_int
        L.orc_lattice_run.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64,
                                      ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_int, u16p, f64p, i64p, i64p, u8p, u8p, f64p]
        L.orc_lattice_run.restype = None
        L.orc_offlattice_run.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, f64p, f64p, f64p,
                                         u8p, u8p, f64p]
        L.orc_offlattice_run.restype = None
        L.orc_lattice_run_restart.argtypes = [
            ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
            ctypes.c_double, ctypes.c_int, ctypes.c_int, u16p, f64p, i64p, i64p, u8p, u8p, f64p,
            u32p]
        L.orc_lattice_run_restart.restype = None
        L.orc_offlattice_run_restart.argtypes = [
            ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
            ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_int, ctypes.c_int, f64p, f64p, f64p, u8p, u8p, f64p, u32p]
        L.orc_offlattice_run_restart.restype = None
        L.orc_reduce.argtypes = [ctypes.c_int64, f64p, f64p, f64p, ctypes.c_int,
                                 ctypes.c_int, f64p]
        L.orc_reduce.restype = None
        L.orc_reduce_n.argtypes = [ctypes.c_int64, f64p, f64p, f64p, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_double, f64p]
        L.orc_reduce_n.restype = None
        L.orc_enumerate.argtypes = [ctypes.c_int, i64p, i64p, i64p]
        L.orc_enumerate.restype = ctypes.c_int
        L.orc_perm_run.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double, i64p,
                                   f64p, f64p, i64p, f64p, i32p, i32p]
        L.orc_perm_run.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def default_threads():
    return max(1, len(os.sched_getaffinity(0)))


def philox4x32_10(ctr, key):
    """Philox4x32-10 of a 4-word counter under a 2-word key (SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                            _ptr(out, ctypes.c_uint32))
    return out


def lattice_run(seed, N, C, beta_eps=0.0, ensemble=0, chain0=0, threads=None,
                trace=False, coords=False, max_attempts=1):
    """Grow chains chain0 .. chain0+C-1 on the cubic lattice (Algorithm 1, Eq. 3).

    Returns a dict of numpy arrays: counts [C,8] u16, logw [C] f64, r2 [C] i64,
    n2rg2 [C] i64, alive [C] u8, attempts [C] u32, and optionally
    trace [C,N-1] u8 and coords [C,N,3] f64.  max_attempts > 1 selects restart
    mode (Section 3.3.2: a trapped chain is grown again from the start).
    """
    C = int(C)
    out = {
        "counts": np.zeros((C, 8), np.uint16),
        "logw": np.zeros(C, np.float64),
        "r2": np.zeros(C, np.int64),
        "n2rg2": np.zeros(C, np.int64),
        "alive": np.zeros(C, np.uint8),
        "attempts": np.zeros(C, np.uint32),
    }
    if trace:
        out["trace"] = np.zeros((C, N - 1), np.uint8)
    if coords:
        out["coords"] = np.zeros((C, N, 3), np.float64)
    lib().orc_lattice_run_restart(
        int(seed), int(ensemble), int(chain0), C, int(N), float(beta_eps), int(max_attempts),
        int(threads or default_threads()),
        _ptr(out["counts"], ctypes.c_uint16), _ptr(out["logw"], ctypes.c_double),
        _ptr(out["r2"], ctypes.c_int64), _ptr(out["n2rg2"], ctypes.c_int64),
        _ptr(out["alive"], ctypes.c_uint8), _ptr(out.get("trace"), ctypes.c_uint8),
        _ptr(out.get("coords"), ctypes.c_double), _ptr(out["attempts"], ctypes.c_uint32))
    return out


def offlattice_run(seed, N, C, k, potential=HARD_SPHERE, beta_eps=0.0, sigma=1.0,
                   cutoff=2.5, ensemble=0, chain0=0, threads=None, trace=False,
                   coords=False, max_attempts=1):
    """Grow chains in real space with k trials per step (Algorithm 2).

    Returns logw [C], r2 [C], rg2 [C] (f64), alive [C] u8, attempts [C] u32 and
    optionally trace [C,N-1] u8 and coords [C,N,3] f64.  max_attempts > 1
    selects restart mode (Section 3.3.3).
    """
    C = int(C)
    out = {
        "logw": np.zeros(C, np.float64),
        "r2": np.zeros(C, np.float64),
        "rg2": np.zeros(C, np.float64),
        "alive": np.zeros(C, np.uint8),
        "attempts": np.zeros(C, np.uint32),
    }
    if trace:
        out["trace"] = np.zeros((C, N - 1), np.uint8)
    if coords:
        out["coords"] = np.zeros((C, N, 3), np.float64)
    lib().orc_offlattice_run_restart(
        int(seed), int(ensemble), int(chain0), C, int(N), int(k), int(potential),
        float(sigma), float(cutoff), float(beta_eps), int(max_attempts),
        int(threads or default_threads()),
        _ptr(out["logw"], ctypes.c_double), _ptr(out["r2"], ctypes.c_double),
        _ptr(out["rg2"], ctypes.c_double), _ptr(out["alive"], ctypes.c_uint8),
        _ptr(out.get("trace"), ctypes.c_uint8), _ptr(out.get("coords"), ctypes.c_double),
        _ptr(out["attempts"], ctypes.c_uint32))
    return out


STAT_KEYS = ["n", "n_alive", "log_max", "S0", "S1", "S2", "Q0", "Q1_r2", "Q2_r2",
             "Q1_rg2", "Q2_rg2", "logZ", "logZ_norm", "mean_r2", "se_r2", "mean_rg2",
             "se_rg2", "ess"]


def reduce(logw, A1, A2, N, k=0, n=None):
    """W-weighted ensemble statistics (Eq. 2 with W as the importance weight, Eq. 9).

    n is Eq. 9's sample size: the number of chains (default) or, in restart
    mode, the number of growth attempts made.
    """
    lw = np.ascontiguousarray(logw, dtype=np.float64)
    a = np.ascontiguousarray(A1, dtype=np.float64)
    b = np.ascontiguousarray(A2, dtype=np.float64)
    out = np.zeros(len(STAT_KEYS), np.float64)
    if n is None:
        lib().orc_reduce(len(lw), _ptr(lw, ctypes.c_double), _ptr(a, ctypes.c_double),
                         _ptr(b, ctypes.c_double), int(N), int(k), _ptr(out, ctypes.c_double))
    else:
        lib().orc_reduce_n(len(lw), _ptr(lw, ctypes.c_double), _ptr(a, ctypes.c_double),
                           _ptr(b, ctypes.c_double), int(N), int(k), float(n),
                           _ptr(out, ctypes.c_double))
    return dict(zip(STAT_KEYS, out.tolist()))


def lattice_logw_from_counts(counts):
    """log W of an athermal lattice chain from its factor counts: sum_m counts[m] log m."""
    counts = np.asarray(counts, dtype=np.float64)
    logs = np.array([-np.inf, 0.0, np.log(2), np.log(3), np.log(4), np.log(5), np.log(6),
                     0.0])
    with np.errstate(invalid="ignore"):
        lw = (counts[:, 1:7] * logs[1:7]).sum(axis=1)
    lw[counts[:, 0] > 0] = -np.inf
    return lw


def enumerate_saw(nmax):
    """Exact cubic-lattice SAW enumeration up to nmax steps.

    Returns (cnt, sr2, sg2), int64 arrays of shape (nmax+1, nmax+1), row = steps n,
    column = number of non-bonded nearest-neighbour contacts: the number of walks,
    their summed R_ee^2 and their summed (n+1)^2 R_g^2.
    """
    shape = (nmax + 1, nmax + 1)
    cnt = np.zeros(shape, np.int64)
    sr2 = np.zeros(shape, np.int64)
    sg2 = np.zeros(shape, np.int64)
    rc = lib().orc_enumerate(int(nmax), _ptr(cnt, ctypes.c_int64), _ptr(sr2, ctypes.c_int64),
                             _ptr(sg2, ctypes.c_int64))
    if rc != 0:
        raise ValueError("nmax out of range")
    return cnt, sr2, sg2


def perm_run(seed, N, M0, max_pop=None, beta_eps=0.0, mu=4.684, c_hi=3.0, c_lo=1.0 / 3.0,
             ensemble=0, positions=False):
    """Breadth-first PERM on the cubic lattice (pruned-enriched Rosenbluth
    growth; Grassberger, Phys. Rev. E 56, 3682 (1997)): a population of M0
    chains grows step by step; after step i a chain with W > c_hi mu^i is
    enriched (two copies sharing W), one with W < c_lo mu^i is pruned (kept
    with probability 1/2 with 2W), within a population cap max_pop.

    Returns pop [N] (population after each step), logz [N] (log of Eq. 9's
    estimate of Z_i from the chains grown at step i), r2 [N] (their
    W-weighted <R_ee^2>), and the final population: w_m, w_e (W = w_m 2^w_e)
    and, with positions, pos [n, N, 3].
    """
    max_pop = int(max_pop or 4 * M0)
    pop = np.zeros(N, np.int64)
    logz = np.zeros(N, np.float64)
    r2 = np.zeros(N, np.float64)
    fn = np.zeros(1, np.int64)
    w_m = np.zeros(max_pop, np.float64)
    w_e = np.zeros(max_pop, np.int32)
    pos = np.zeros((max_pop, N, 3), np.int32) if positions else None
    rc = lib().orc_perm_run(int(seed), int(ensemble), int(N), float(beta_eps), int(M0),
                            int(max_pop), float(mu), float(c_hi), float(c_lo),
                            _ptr(pop, ctypes.c_int64), _ptr(logz, ctypes.c_double),
                            _ptr(r2, ctypes.c_double), _ptr(fn, ctypes.c_int64),
                            _ptr(w_m, ctypes.c_double), _ptr(w_e, ctypes.c_int32),
                            _ptr(pos, ctypes.c_int32))
    if rc != 0:
        raise ValueError("perm_run: bad arguments")
    n = int(fn[0])
    out = {"pop": pop, "logz": logz, "r2": r2, "n": n, "w_m": w_m[:n], "w_e": w_e[:n]}
    if positions:
        out["pos"] = pos[:n]
    return out
