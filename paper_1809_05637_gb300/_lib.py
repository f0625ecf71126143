"""ctypes binding of libdclno (include/dclno.h).  Marshalling only."""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdclno.so")

DCLNO_FP64 = 0
DCLNO_MIXED = 1
DCLNO_LNO_PAPER = 0
DCLNO_LNO_SYM = 1
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_NOT_SPD", 5: "ERR_NO_BRACKET",
                6: "ERR_NOT_CONVERGED", 7: "ERR_TIMEOUT", 8: "ERR_NO_LNOS"}

# every entry point declared in include/dclno.h
SYMBOLS = ["dclno_create", "dclno_destroy", "dclno_last_error", "dclno_build_clusters", "dclno_compute_lnos",
           "dclno_solve_clusters", "dclno_find_mu", "dclno_density_matrix", "dclno_step", "dclno_cluster_info",
           "dclno_get_spectrum", "dclno_get_lnos", "dclno_launch_count", "dclno_set_profiling",
           "dclno_kernel_time", "dclno_measure_fp64_peaks", "dclno_find_mu_noalloc", "dclno_scf_run",
           "dclno_density_matrices", "dclno_set_workspace_limit", "dclno_batch_info",
           "dclno_set_autotune", "dclno_get_tuning", "dclno_build_clusters_kappa", "dclno_set_lno_threshold",
           "dclno_get_lno_counts", "dclno_set_lno_mode", "dclno_set_tridiag", "dclno_density_matrix_poles",
           "dclno_set_mixed_engine", "dclno_set_schedule", "dclno_set_tuning_cache", "dclno_tuning_report",
           "dclno_set_bucket_min", "dclno_set_tear", "dclno_refine_eigenpairs"]


class DclnoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class dclno_system(ctypes.Structure):
    _fields_ = [
        ("natoms", ctypes.c_int),
        ("pos", ctypes.c_void_p),
        ("cell", ctypes.c_void_p),
        ("pbc", ctypes.c_void_p),
        ("norb", ctypes.c_void_p),
        ("nnzb", ctypes.c_longlong),
        ("nval", ctypes.c_longlong),
        ("row_ptr", ctypes.c_void_p),
        ("col", ctypes.c_void_p),
        ("shift", ctypes.c_void_p),
        ("blk_off", ctypes.c_void_p),
        ("H", ctypes.c_void_p),
        ("S", ctypes.c_void_p),
    ]


_LIB = None


def load_library():
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    sigs = {
        "dclno_create": ([ctypes.POINTER(P), P], I),
        "dclno_destroy": ([P], None),
        "dclno_last_error": ([P], ctypes.c_char_p),
        "dclno_build_clusters": ([P, ctypes.POINTER(dclno_system), D, D, I], I),
        "dclno_compute_lnos": ([P, P], I),
        "dclno_solve_clusters": ([P, I], I),
        "dclno_find_mu": ([P, D, D, P, P], I),
        "dclno_density_matrix": ([P, D, D, P, P], I),
        "dclno_step": ([P, P, P, I, I, D, D, P, P, P], I),
        "dclno_cluster_info": ([P, P, P, P], I),
        "dclno_get_spectrum": ([P, P, P], I),
        "dclno_get_lnos": ([P, P, P, P, P], I),
        "dclno_launch_count": ([P], ctypes.c_longlong),
        "dclno_set_profiling": ([P, I], I),
        "dclno_kernel_time": ([P, ctypes.c_char_p, P, P], I),
        "dclno_measure_fp64_peaks": ([P, P], I),
        "dclno_find_mu_noalloc": ([P, P, ctypes.c_longlong, D, D, P, P, P], I),
        "dclno_scf_run": ([P, P, I, D, I, D, D, I, P, P, P], I),
        "dclno_density_matrices": ([P, D, D, P, P, P], I),
        "dclno_set_workspace_limit": ([P, ctypes.c_size_t], I),
        "dclno_batch_info": ([P, P, P], I),
        "dclno_set_autotune": ([P, I], I),
        "dclno_get_tuning": ([P, I, P, P], I),
        "dclno_build_clusters_kappa": ([P, ctypes.POINTER(dclno_system), D, I, D, D], I),
        "dclno_set_lno_threshold": ([P, I, D], I),
        "dclno_set_lno_mode": ([P, I], I),
        "dclno_get_lno_counts": ([P, P], I),
        "dclno_set_tridiag": ([P, I], I),
        "dclno_density_matrix_poles": ([P, D, D, I, I, P], I),
        "dclno_set_mixed_engine": ([P, I], I),
        "dclno_set_schedule": ([P, I], I),
        "dclno_set_bucket_min": ([P, I], I),
        "dclno_set_tear": ([P, I], I),
        "dclno_set_tuning_cache": ([P, ctypes.c_char_p], I),
        "dclno_tuning_report": ([P, ctypes.c_char_p, ctypes.c_size_t, P], I),
        "dclno_refine_eigenpairs": ([P, P, P, P, I, I, I, P], I),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _LIB = lib
    return lib


def exported_symbols():
    """Names of SYMBOLS that the built library exports."""
    lib = load_library()
    return [s for s in SYMBOLS if hasattr(lib, s)]


def measure_fp64_peaks():
    """(DFMA, DMMA) FP64 TFLOP/s of the current CUDA device, measured now."""
    lib = load_library()
    a, b = ctypes.c_double(), ctypes.c_double()
    st = lib.dclno_measure_fp64_peaks(_dptr(a), _dptr(b))
    if st != 0:
        raise DclnoError(st, "dclno_measure_fp64_peaks failed")
    return a.value, b.value


def find_mu_noalloc(eps, q, n_electrons, kT, stream=None):
    """dclno_find_mu_noalloc on device arrays eps, q (torch, float64); returns (mu, N(mu)).

    The library allocates nothing in this call (see include/dclno.h).  The C entry
    point reads `count` doubles from each pointer and cannot check them, so the
    arrays are checked here: contiguous torch.float64 CUDA tensors of the same
    length on the current device."""
    import torch

    lib = load_library()
    for name, t in (("eps", eps), ("q", q)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError(f"find_mu_noalloc: {name} must be a contiguous torch.float64 CUDA tensor")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"find_mu_noalloc: {name} is on {t.device}, not on the current device "
                             f"cuda:{torch.cuda.current_device()}")
    if eps.numel() != q.numel():
        raise ValueError(f"find_mu_noalloc: eps has {eps.numel()} elements, q has {q.numel()}")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    mu, n = ctypes.c_double(), ctypes.c_double()
    st = lib.dclno_find_mu_noalloc(_ptr(eps), _ptr(q), int(eps.numel()), float(n_electrons), float(kT),
                                   _dptr(mu), _dptr(n), ctypes.c_void_p(stream))
    if st != 0:
        raise DclnoError(st, "dclno_find_mu_noalloc failed")
    return mu.value, n.value


def refine_eigenpairs(H, S, X, nsweeps=1, stream=None):
    """dclno_refine_eigenpairs on a batch of pencils: H, S, X are [count, n, n] float64
    CUDA tensors (X updated in place); returns the eigenvalue estimates of the last
    sweep as a [count, n] tensor."""
    import torch

    lib = load_library()
    dev = torch.cuda.current_device()
    for name, t in (("H", H), ("S", S), ("X", X)):
        if not isinstance(t, torch.Tensor) or t.dim() != 3 or t.shape[1] != t.shape[2]:
            raise ValueError(f"refine_eigenpairs: {name} must be a [count, n, n] torch tensor")
        _require_doubles(name, t, t.numel(), "device", dev)
    if not (H.shape == S.shape == X.shape):
        raise ValueError(f"refine_eigenpairs: shapes differ: H {tuple(H.shape)}, S {tuple(S.shape)}, X {tuple(X.shape)}")
    count, n = int(X.shape[0]), int(X.shape[1])
    lam = torch.empty((count, n), dtype=torch.float64, device=X.device)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = lib.dclno_refine_eigenpairs(_ptr(H), _ptr(S), _ptr(X), _ptr(lam), n, count, int(nsweeps),
                                     ctypes.c_void_p(stream))
    if st != 0:
        raise DclnoError(st, "dclno_refine_eigenpairs failed")
    return lam


def _ptr(x):
    """Address of a numpy array (host) or a torch tensor (device or host)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _require_doubles(name, x, count, where, device=None):
    """Refuse a buffer that the C library would read or write past: it must hold at
    least `count` contiguous float64 values, on CUDA device `device` (where="device":
    a torch tensor) or in host memory (where="host": a numpy array or a CPU tensor).
    The C entry points receive bare pointers and cannot check any of this."""
    if isinstance(x, np.ndarray):
        ok = where == "host" and x.dtype == np.float64 and x.flags.c_contiguous
        n = x.size
    else:
        import torch

        if not isinstance(x, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor or a numpy array, not {type(x).__name__}")
        on_gpu = x.is_cuda
        ok = x.dtype == torch.float64 and x.is_contiguous() and (
            (where == "device" and on_gpu and x.device.index == device) or (where == "host" and not on_gpu))
        n = x.numel()
    if not ok:
        at = f"CUDA tensor on cuda:{device}" if where == "device" else "host array"
        raise ValueError(f"{name} must be a contiguous float64 {at}")
    if n < count:
        raise ValueError(f"{name} holds {n} values; the system's H, S and rho hold {count}")


def _dptr(v: ctypes.c_double):
    return ctypes.cast(ctypes.byref(v), ctypes.c_void_p)


class Context:
    """One libdclno context bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream=None):
        self.lib = load_library()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        import torch

        h = ctypes.c_void_p()
        self._check(self.lib.dclno_create(ctypes.byref(h), ctypes.c_void_p(stream)), None)
        self.h = h
        self.device = torch.cuda.current_device()  # the device dclno_create bound the context to
        self._keep = []
        self.natoms = 0
        self.nval = 0

    def _check(self, st, h="self"):
        if st != 0:
            msg = self.lib.dclno_last_error(self.h if h == "self" else None)
            raise DclnoError(st, (msg or b"").decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.dclno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_workspace_limit(self, nbytes):
        """Workspace budget in bytes for the next build_clusters (0 = free device memory)."""
        self._check(self.lib.dclno_set_workspace_limit(self.h, ctypes.c_size_t(int(nbytes))))

    def batch_info(self):
        """(number of memory-admitted batches, workspace arena bytes) after build_clusters."""
        nb, ws = ctypes.c_int(), ctypes.c_size_t()
        self._check(self.lib.dclno_batch_info(self.h, ctypes.cast(ctypes.byref(nb), ctypes.c_void_p),
                                              ctypes.cast(ctypes.byref(ws), ctypes.c_void_p)))
        return nb.value, ws.value

    def set_lno_threshold(self, lambda_th):
        """Keep the LNOs with eigenvalue >= lambda_th (at most k_lno per atom); None = fixed k_lno."""
        on = lambda_th is not None
        self._check(self.lib.dclno_set_lno_threshold(self.h, int(on), float(lambda_th) if on else 0.0))

    def set_lno_mode(self, mode):
        """DCLNO_LNO_PAPER (Lambda_0i, the default) or DCLNO_LNO_SYM ((S rho S)_ii v = lambda S_ii v)."""
        self._check(self.lib.dclno_set_lno_mode(self.h, int(mode)))

    def lno_counts(self):
        """LNOs per atom of the last LNO computation."""
        k = np.zeros(self.natoms, np.int32)
        self._check(self.lib.dclno_get_lno_counts(self.h, _ptr(k)))
        return k

    def set_tridiag(self, mode):
        """Tridiagonalisation form: 0 automatic, 1 one-stage, 2 two-stage (dense -> band -> tridiagonal)."""
        self._check(self.lib.dclno_set_tridiag(self.h, int(mode)))

    def set_mixed_engine(self, engine):
        """Engine of the mixed path's K <= 32 tile products: 0 tuned, 1 mma.sync, 2 tcgen05."""
        self._check(self.lib.dclno_set_mixed_engine(self.h, int(engine)))

    def set_schedule(self, mode):
        """Grid form of the cubic kernels: 0 tuned, 1 one CTA per cluster, 2 persistent."""
        self._check(self.lib.dclno_set_schedule(self.h, int(mode)))

    def set_tear(self, mode):
        """Cuppen's tear: 0 automatic (twice from dimension 512), 1 once, 2 twice (from 64); before the build."""
        self._check(self.lib.dclno_set_tear(self.h, int(mode)))

    def set_bucket_min(self, count):
        """Minimum clusters per size bucket (0: twice the SM count; 1: every 64-wide bucket)."""
        self._check(self.lib.dclno_set_bucket_min(self.h, int(count)))

    def set_tuning_cache(self, path):
        """Text cache of tuned schedules (None: off)."""
        self._check(self.lib.dclno_set_tuning_cache(self.h, None if path is None else str(path).encode()))

    def tuning_report(self):
        """Size buckets and their schedules, as a dict."""
        import json

        need = ctypes.c_size_t()
        self._check(self.lib.dclno_tuning_report(self.h, None, 0, ctypes.cast(ctypes.byref(need), ctypes.c_void_p)))
        buf = ctypes.create_string_buffer(need.value)
        self._check(self.lib.dclno_tuning_report(self.h, buf, need.value, None))
        return json.loads(buf.value.decode())

    def set_autotune(self, on=True):
        """Time the QL launch shape on each batch's first eager solve (default on)."""
        self._check(self.lib.dclno_set_autotune(self.h, int(bool(on))))

    def tuning(self, batch=0):
        """(QL lanes per warp chosen for `batch` (0 = not tuned), timed ms of the candidates
        4, 8, 12, 16, 24, 32 lanes (-1 = not tried))."""
        lanes = ctypes.c_int()
        ms = np.zeros(6, np.float32)
        self._check(self.lib.dclno_get_tuning(self.h, int(batch), ctypes.cast(ctypes.byref(lanes), ctypes.c_void_p),
                                              _ptr(ms)))
        return lanes.value, ms

    # ---- the five calls of a DC-LNO step
    def build_clusters(self, pos, cell, pbc, norb, row_ptr, col, shift, blk_off, H, S, r_core, r_lno, k_lno,
                       kappa=None, s_fna=0.0):
        """Truncated clusters with a fixed short-range radius r_core, or with the
        paper's region rule (kappa, s_fna given; r_core is then ignored)."""
        host = dict(
            pos=np.ascontiguousarray(pos, dtype=np.float64), cell=np.ascontiguousarray(cell, dtype=np.float64),
            pbc=np.ascontiguousarray(np.asarray(pbc).astype(np.int32)),
            norb=np.ascontiguousarray(norb, dtype=np.int32), row_ptr=np.ascontiguousarray(row_ptr, dtype=np.int64),
            col=np.ascontiguousarray(col, dtype=np.int32), shift=np.ascontiguousarray(shift, dtype=np.int8),
            blk_off=np.ascontiguousarray(blk_off, dtype=np.int64))
        _require_doubles("H", H, 0, "device", self.device)
        nval = int(H.numel())
        _require_doubles("S", S, nval, "device", self.device)
        s = dclno_system(natoms=len(host["norb"]), pos=_ptr(host["pos"]), cell=_ptr(host["cell"]),
                         pbc=_ptr(host["pbc"]), norb=_ptr(host["norb"]), nnzb=len(host["col"]), nval=nval,
                         row_ptr=_ptr(host["row_ptr"]), col=_ptr(host["col"]), shift=_ptr(host["shift"]),
                         blk_off=_ptr(host["blk_off"]), H=_ptr(H), S=_ptr(S))
        if kappa is None:
            self._check(self.lib.dclno_build_clusters(self.h, ctypes.byref(s), float(r_core), float(r_lno),
                                                      int(k_lno)))
        else:
            self._check(self.lib.dclno_build_clusters_kappa(self.h, ctypes.byref(s), float(r_lno), int(k_lno),
                                                            float(kappa), float(s_fna)))
        self._keep = [H, S]
        self.natoms = len(host["norb"])
        self.nval = nval
        self.norb = host["norb"]
        self.k_lno = int(k_lno)

    def _dev(self, name, x):
        """A device buffer of the system's nval values (None passes through)."""
        if x is not None:
            _require_doubles(name, x, self.nval, "device", self.device)
        return _ptr(x)

    def compute_lnos(self, rho):
        """LNOs from rho (device, nval values); rho None: the first step's LNO-free start."""
        self._dev("rho", rho)
        self._check(self.lib.dclno_compute_lnos(self.h, _ptr(rho)))

    def solve_clusters(self, precision=DCLNO_FP64):
        self._check(self.lib.dclno_solve_clusters(self.h, int(precision)))

    def find_mu(self, n_electrons, kT):
        mu, n = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.dclno_find_mu(self.h, float(n_electrons), float(kT), _dptr(mu), _dptr(n)))
        return mu.value, n.value

    def density_matrix(self, mu, kT, rho_out):
        e = ctypes.c_double()
        self._dev("rho_out", rho_out)
        self._check(self.lib.dclno_density_matrix(self.h, float(mu), float(kT), _ptr(rho_out), _dptr(e)))
        return e.value

    def density_matrix_poles(self, mu, kT, n_poles, rho_out, precision=DCLNO_FP64):
        """rho rows from the Matsubara pole sum (no eigenvectors); invalidates an earlier solve."""
        self._dev("rho_out", rho_out)
        self._check(self.lib.dclno_density_matrix_poles(self.h, float(mu), float(kT), int(n_poles), int(precision),
                                                        _ptr(rho_out)))

    def density_matrices(self, mu, kT, rho_out, edm_out):
        """rho and the energy density matrix e (Eq. (edm)) rows; returns the band energy."""
        e = ctypes.c_double()
        self._dev("rho_out", rho_out)
        self._dev("edm_out", edm_out)
        self._check(self.lib.dclno_density_matrices(self.h, float(mu), float(kT), _ptr(rho_out), _ptr(edm_out),
                                                    _dptr(e)))
        return e.value

    def step(self, rho_in, rho_out, n_electrons, kT, host_buffers=False, precision=DCLNO_FP64):
        mu, n, e = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        for name, x in (("rho_in", rho_in), ("rho_out", rho_out)):
            if x is not None:
                _require_doubles(name, x, self.nval, "host" if host_buffers else "device", self.device)
        self._check(self.lib.dclno_step(self.h, _ptr(rho_in), _ptr(rho_out), int(bool(host_buffers)),
                                        int(precision), float(n_electrons), float(kT), _dptr(mu), _dptr(n),
                                        _dptr(e)))
        return mu.value, n.value, e.value

    def scf_run(self, rho, nsteps, alpha, n_electrons, kT, precision=DCLNO_FP64, use_graph=False):
        """nsteps of (DC-LNO step, rho <- rho + alpha (rho_out - rho)) on the device array rho.

        Returns per-step (mu, N(mu), E_band) as numpy arrays."""
        mu = np.zeros(nsteps)
        n = np.zeros(nsteps)
        e = np.zeros(nsteps)
        self._dev("rho", rho)
        self._check(self.lib.dclno_scf_run(self.h, _ptr(rho), int(nsteps), float(alpha), int(precision),
                                           float(n_electrons), float(kT), int(bool(use_graph)), _ptr(mu),
                                           _ptr(n), _ptr(e)))
        return mu, n, e

    # ---- inspection
    def cluster_info(self):
        dims = np.zeros(self.natoms, np.int32)
        nmem = np.zeros(self.natoms, np.int32)
        tot = ctypes.c_longlong()
        self._check(self.lib.dclno_cluster_info(self.h, _ptr(dims), _ptr(nmem),
                                                ctypes.cast(ctypes.byref(tot), ctypes.c_void_p)))
        return dims, nmem, tot.value

    def spectrum(self):
        dims, _, tot = self.cluster_info()
        eps = np.zeros(tot)
        q = np.zeros(tot)
        self._check(self.lib.dclno_get_spectrum(self.h, _ptr(eps), _ptr(q)))
        off = np.concatenate([[0], np.cumsum(dims)])
        return [(eps[off[i]:off[i + 1]], q[off[i]:off[i + 1]]) for i in range(self.natoms)]

    def lnos(self):
        k = self.k_lno
        V = np.zeros(int(np.sum(self.norb)) * k)
        lre = np.zeros(int(np.sum(self.norb)))
        lim = np.zeros_like(lre)
        fl = np.zeros(self.natoms, np.int32)
        self._check(self.lib.dclno_get_lnos(self.h, _ptr(V), _ptr(lre), _ptr(lim), _ptr(fl)))
        out = {}
        vo = mo = 0
        for i, m in enumerate(self.norb):
            m = int(m)
            out[i] = (V[vo:vo + m * k].reshape(m, k), lre[mo:mo + m] + 1j * lim[mo:mo + m], int(fl[i]))
            vo += m * k
            mo += m
        return out

    def launch_count(self):
        return int(self.lib.dclno_launch_count(self.h))

    def set_profiling(self, on=True):
        self._check(self.lib.dclno_set_profiling(self.h, int(bool(on))))

    def kernel_time(self, name):
        """(total milliseconds, launches) of kernel `name` since profiling was switched on."""
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        self._check(self.lib.dclno_kernel_time(self.h, name.encode(), _dptr(ms),
                                               ctypes.cast(ctypes.byref(n), ctypes.c_void_p)))
        return ms.value, n.value
