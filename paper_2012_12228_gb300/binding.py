"""ctypes binding of the C ABI in include/ftq.h (argument marshalling only).

Device buffers are torch tensors; the binding passes their data pointers and
the current CUDA stream.  Every call checks the returned status and raises
``FTQError`` with the library's message.
"""
import ctypes
import math
import os

FTQ_FP64, FTQ_MIXED, FTQ_MIXED_SIMT, FTQ_MIXED_F64UDT = 0, 1, 2, 3
FTQ_PHASELESS, FTQ_FREE = 0, 1
FTQ_OVERLAP_PAPER, FTQ_OVERLAP_MODIFIED = 0, 1
_Q = dict(M=0, N_ALPHA=1, N_SLICES=2, SLICE=3, WALKERS=4, NCUT2=5, PRECISION=6, DEVICE_BYTES=7, QR_PANEL=8,
          GREEN_KERNEL=9)
_F = dict(BETA=0, DTAU=1, MU=2, MU_T=3, L=4, E_M=5)

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


class FTQError(RuntimeError):
    pass


class Opts(ctypes.Structure):
    _fields_ = [("walkers", ctypes.c_int), ("stabilise_every", ctypes.c_int),
                ("exp_order", ctypes.c_int), ("precision", ctypes.c_int),
                ("constraint", ctypes.c_int), ("overlap", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("cuda_stream", ctypes.c_void_p),
                ("force_bias_cap", ctypes.c_double), ("low_rank_threshold", ctypes.c_double)]


class System(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int), ("rs", ctypes.c_double), ("theta", ctypes.c_double),
                ("mu", ctypes.c_double), ("dtau", ctypes.c_double), ("walkers", ctypes.c_int),
                ("reserved", ctypes.c_int)]


EXPORTS = ["ftq_init_ueg", "ftq_reset", "ftq_propagate_slices", "ftq_stabilise", "ftq_green",
           "ftq_estimators", "ftq_weights", "ftq_status", "ftq_query", "ftq_query_f64",
           "ftq_basis", "ftq_transfers", "ftq_profile", "ftq_profile_read", "ftq_estimators_noalloc", "ftq_mu_grad",
           "ftq_init_batch", "ftq_batch_member", "ftq_batch_propagate", "ftq_autotune", "ftq_fields", "ftq_population_control", "ftq_structure_factor", "ftq_pair_branch",
           "ftq_ranks", "ftq_set_wait_limit", "ftq_set_green_kernel", "ftq_track_estimates", "ftq_slice_estimates",
           "ftq_last_error", "ftq_destroy"]
KERNELS = {"force_bias": 0, "chain": 1, "qrcp": 2, "green": 3, "estimators": 4, "init": 5, "bridge": 6,
           "border": 7, "fields": 8, "population": 9, "tinv": 10}
K_COUNT = 11


def library_path():
    return os.path.join(HERE, "_build", "libftq.so")


def load_library(path=None):
    """Load libftq.so (built by ``paper_2012_12228_gb300.build``); raises if absent."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or library_path()
    if not os.path.exists(p):
        raise FTQError(f"{p} not found: run __graft_entry__.build() (nvcc, sm_103a) first")
    lib = ctypes.CDLL(p)
    vp, i, d, i64p, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
    lib.ftq_init_ueg.argtypes = [ctypes.POINTER(vp), i, i, d, d, d, d, ctypes.POINTER(Opts)]
    lib.ftq_reset.argtypes = [vp]
    lib.ftq_propagate_slices.argtypes = [vp, i, vp]
    lib.ftq_stabilise.argtypes = [vp]
    lib.ftq_green.argtypes = [vp, vp]
    lib.ftq_estimators.argtypes = [vp, dp, vp]
    lib.ftq_weights.argtypes = [vp, vp]
    lib.ftq_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    lib.ftq_ranks.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    lib.ftq_set_wait_limit.argtypes = [vp, ctypes.c_int64]
    lib.ftq_set_green_kernel.argtypes = [vp, i]
    lib.ftq_track_estimates.argtypes = [vp, i]
    lib.ftq_slice_estimates.argtypes = [vp, dp, i]
    lib.ftq_query.argtypes = [vp, i, i64p]
    lib.ftq_query_f64.argtypes = [vp, i, dp]
    lib.ftq_basis.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
    lib.ftq_transfers.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
    lib.ftq_profile.argtypes = [vp, i]
    lib.ftq_profile_read.argtypes = [vp, dp, i64p]
    lib.ftq_estimators_noalloc.argtypes = [i, i, d, vp, i, vp, vp]
    lib.ftq_mu_grad.argtypes = [vp, dp, vp]
    lib.ftq_init_batch.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(System), ctypes.POINTER(Opts)]
    lib.ftq_batch_member.argtypes = [vp, i, ctypes.POINTER(vp)]
    lib.ftq_batch_propagate.argtypes = [vp, i, ctypes.POINTER(vp)]
    lib.ftq_autotune.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]
    lib.ftq_fields.argtypes = [vp, i, i, vp]
    lib.ftq_population_control.argtypes = [vp, d, vp]
    lib.ftq_structure_factor.argtypes = [vp, dp, vp]
    lib.ftq_pair_branch.argtypes = [vp, dp, vp]
    lib.ftq_last_error.argtypes = [vp]
    lib.ftq_last_error.restype = ctypes.c_char_p
    lib.ftq_destroy.argtypes = [vp]
    lib.ftq_destroy.restype = None
    for name in EXPORTS[:-2]:
        if name != "ftq_last_error":
            getattr(lib, name).restype = ctypes.c_int
    if path is None:
        _LIB = lib
    return lib


class Propagator:
    """One UEG system with W walkers on the current CUDA device.

    Parameters mirror ftq_init_ueg and ftq_opts; ``mu=None`` selects
    mu = mu_T; ``overlap`` is FTQ_OVERLAP_PAPER (S_k, Eq. ftoratio) or
    FTQ_OVERLAP_MODIFIED (S~_k, Eq. ztfix); ``low_rank`` > 0 is the
    truncation threshold of Eq. thresh (complex128 path only)."""

    def __init__(self, N, M, rs, theta, dtau, mu=None, walkers=64, stabilise_every=5,
                 exp_order=6, precision=FTQ_FP64, constraint=FTQ_PHASELESS, seed=0, stream=None,
                 overlap=FTQ_OVERLAP_PAPER, low_rank=0.0):
        import torch
        if not torch.cuda.is_available():
            raise FTQError("no CUDA device: the propagator has no CPU path")
        self._torch = torch
        self.lib = load_library()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        o = Opts(walkers, stabilise_every, exp_order, precision, constraint, overlap, seed,
                 ctypes.c_void_p(self.stream.cuda_stream), 0.0, float(low_rank))
        h = ctypes.c_void_p()
        st = self.lib.ftq_init_ueg(ctypes.byref(h), N, M, rs, theta,
                                   float("nan") if mu is None else float(mu), dtau, ctypes.byref(o))
        if st != 0:
            raise FTQError(f"ftq_init_ueg: {self.lib.ftq_last_error(None).decode()} (status {st})")
        self.h = h
        self.N = N
        self.W = walkers
        self.M = self.query("M")
        self.n_alpha = self.query("N_ALPHA")
        self.n_slices = self.query("N_SLICES")

    @classmethod
    def _member(cls, lib, handle, walkers):
        """Non-owning view of a batch member context."""
        import torch
        obj = cls.__new__(cls)
        obj._torch = torch
        obj.lib = lib
        obj.h = handle
        obj._owned = False
        obj.W = walkers
        obj.M = obj.query("M")
        obj.n_alpha = obj.query("N_ALPHA")
        obj.n_slices = obj.query("N_SLICES")
        return obj

    def autotune(self):
        """Pick the column tiling of the tensor-core chain, the QR panel width and the G(tau)
        kernel by timing; returns (tiles, ms per Horner step)."""
        ch = (ctypes.c_int * 1)()
        ms = (ctypes.c_float * 1)()
        self._check(self.lib.ftq_autotune(self.h, ch, ms), "ftq_autotune")
        return ch[0], ms[0]

    def _check(self, st, what):
        if st != 0:
            raise FTQError(f"{what}: {self.lib.ftq_last_error(self.h).decode()} (status {st})")

    def close(self):
        if getattr(self, "h", None) and getattr(self, "_owned", True):
            self.lib.ftq_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self, key):
        v = ctypes.c_int64()
        self._check(self.lib.ftq_query(self.h, _Q[key], ctypes.byref(v)), "ftq_query")
        return v.value

    def query_f64(self, key):
        v = ctypes.c_double()
        self._check(self.lib.ftq_query_f64(self.h, _F[key], ctypes.byref(v)), "ftq_query_f64")
        return v.value

    def basis(self):
        buf = (ctypes.c_int32 * (3 * self.M))()
        self._check(self.lib.ftq_basis(self.h, buf), "ftq_basis")
        return [tuple(buf[3 * i:3 * i + 3]) for i in range(self.M)]

    def transfers(self):
        n = self.n_alpha // 2
        buf = (ctypes.c_int32 * (3 * n))()
        self._check(self.lib.ftq_transfers(self.h, buf), "ftq_transfers")
        return [tuple(buf[3 * i:3 * i + 3]) for i in range(n)]

    def reset(self):
        self._check(self.lib.ftq_reset(self.h), "ftq_reset")

    def propagate(self, fields):
        """fields: CUDA float64 tensor [n][W][N_alpha] (contiguous), or an int n:
        n slices with the library's own fields (see ``fields``)."""
        t = self._torch
        if isinstance(fields, int):
            self._check(self.lib.ftq_propagate_slices(self.h, fields, None), "ftq_propagate_slices")
            return
        if fields.device.type != "cuda" or fields.dtype != t.float64 or not fields.is_contiguous():
            raise FTQError("fields must be a contiguous CUDA float64 tensor")
        if fields.dim() != 3 or fields.shape[1] != self.W or fields.shape[2] != self.n_alpha:
            raise FTQError(f"fields must have shape [n, {self.W}, {self.n_alpha}]")
        self._check(self.lib.ftq_propagate_slices(self.h, int(fields.shape[0]), ctypes.c_void_p(fields.data_ptr())),
                    "ftq_propagate_slices")

    def fields(self, first_slice, n_slices):
        """The library's own N(0,1) fields of slices [first_slice, first_slice + n_slices)
        (Philox4x32-10 keyed by the seed, Box-Muller): CUDA float64 [n][W][N_alpha]."""
        t = self._torch
        out = t.empty((n_slices, self.W, self.n_alpha), dtype=t.float64, device="cuda")
        self._check(self.lib.ftq_fields(self.h, first_slice, n_slices, ctypes.c_void_p(out.data_ptr())),
                    "ftq_fields")
        return out

    def structure_factor(self, per_walker=False):
        """Weighted <rho(Q) rho(-Q)> and S(Q) = Re <rho(Q) rho(-Q)> / N-bar at the
        current tau for every transfer Q (integer vectors in ``q``, +q and -q of
        each half-space transfer in turn); ``per_walker`` adds the per-walker
        values (CUDA complex128 [W][N_alpha])."""
        import numpy as np
        t = self._torch
        nq = self.n_alpha
        buf = (ctypes.c_double * (4 + 2 * nq))()
        pw = t.empty((self.W, nq), dtype=t.complex128, device="cuda") if per_walker else None
        self._check(self.lib.ftq_structure_factor(self.h, buf, None if pw is None else ctypes.c_void_p(pw.data_ptr())),
                    "ftq_structure_factor")
        vals = np.frombuffer(buf, dtype=np.float64)
        sw = complex(vals[0], vals[1])
        rr = (vals[4::2] + 1j * vals[5::2]) / sw
        qh = (ctypes.c_int32 * (3 * (nq // 2)))()
        self._check(self.lib.ftq_transfers(self.h, qh), "ftq_transfers")
        qh = np.frombuffer(qh, dtype=np.int32).reshape(-1, 3)
        q = np.empty((nq, 3), dtype=np.int32)
        q[0::2], q[1::2] = qh, -qh
        res = {"rhorho": rr, "S": rr.real / self.N, "q": q, "sum_w": sw, "log_scale": vals[2],
               "n_alive": int(vals[3])}
        if pw is not None:
            res["per_walker"] = pw
        return res

    def pair_branch(self, draws):
        """Pair branching with uniform draws in [0, 1) (one per pair, W // 2 of
        them); returns the parent of every slot (CUDA int32 [W])."""
        import numpy as np
        t = self._torch
        d = np.ascontiguousarray(np.asarray(draws, dtype=np.float64)[: self.W // 2])
        if d.size < self.W // 2:
            raise FTQError(f"pair branching needs {self.W // 2} draws")
        parent = t.empty(self.W, dtype=t.int32, device="cuda")
        self._check(self.lib.ftq_pair_branch(self.h, d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             ctypes.c_void_p(parent.data_ptr())), "ftq_pair_branch")
        return parent

    def population_control(self, xi):
        """Comb the walkers with the uniform draw xi in [0, 1); returns the
        parent of every slot (CUDA int32 [W])."""
        t = self._torch
        parent = t.empty(self.W, dtype=t.int32, device="cuda")
        self._check(self.lib.ftq_population_control(self.h, float(xi), ctypes.c_void_p(parent.data_ptr())),
                    "ftq_population_control")
        return parent

    def stabilise(self):
        self._check(self.lib.ftq_stabilise(self.h), "ftq_stabilise")

    def green(self, out=None):
        t = self._torch
        if out is None:
            out = t.empty((self.W, self.M, self.M), dtype=t.complex128, device="cuda")
        self._check(self.lib.ftq_green(self.h, ctypes.c_void_p(out.data_ptr())), "ftq_green")
        return out

    def weights(self):
        t = self._torch
        out = t.empty((self.W, 8), dtype=t.float64, device="cuda")
        self._check(self.lib.ftq_weights(self.h, ctypes.c_void_p(out.data_ptr())), "ftq_weights")
        return out

    def ranks(self):
        """Rank of every walker's right block (numpy int array [W])."""
        import numpy as np
        out = (ctypes.c_int * self.W)()
        self._check(self.lib.ftq_ranks(self.h, out), "ftq_ranks")
        return np.array(out[:], dtype=np.int64)

    def estimators(self, per_walker=True):
        t = self._torch
        pw = t.empty((self.W, 8), dtype=t.float64, device="cuda") if per_walker else None
        buf = (ctypes.c_double * 8)()
        self._check(self.lib.ftq_estimators(self.h, buf, ctypes.c_void_p(pw.data_ptr()) if pw is not None else None),
                    "ftq_estimators")
        sw = complex(buf[0], buf[1])
        res = dict(sum_w=sw, sum_wE=complex(buf[2], buf[3]), sum_wN=complex(buf[4], buf[5]),
                   log_scale=buf[6], n_alive=int(buf[7]))
        res["E"] = res["sum_wE"] / sw if sw != 0 else complex(math.nan, math.nan)
        res["N"] = res["sum_wN"] / sw if sw != 0 else complex(math.nan, math.nan)
        if pw is not None:
            res["per_walker"] = pw
        return res

    def profile(self, enable=True):
        self._check(self.lib.ftq_profile(self.h, 1 if enable else 0), "ftq_profile")

    def profile_read(self):
        """{kernel: (summed event ms of timed launches, launches so far)}"""
        ms = (ctypes.c_double * K_COUNT)()
        n = (ctypes.c_int64 * K_COUNT)()
        self._check(self.lib.ftq_profile_read(self.h, ms, n), "ftq_profile_read")
        return {k: (ms[v], n[v]) for k, v in KERNELS.items()}

    def launches(self):
        return sum(v[1] for v in self.profile_read().values())

    def mu_grad(self, per_walker=True):
        """d<N>/dmu and d<E>/dmu at tau = beta (fixed draws, frozen force bias)."""
        t = self._torch
        pw = t.empty((self.W, 8), dtype=t.float64, device="cuda") if per_walker else None
        buf = (ctypes.c_double * 8)()
        self._check(self.lib.ftq_mu_grad(self.h, buf, ctypes.c_void_p(pw.data_ptr()) if pw is not None else None),
                    "ftq_mu_grad")
        res = dict(dN=buf[0], dE=buf[1], N=buf[2], E=buf[3], n_alive=int(buf[4]), log_scale=buf[5],
                   dN_imag=buf[6], dE_imag=buf[7])
        if pw is not None:
            res["per_walker"] = pw
        return res

    def track_estimates(self, every=1):
        """Record the global estimate after every `every`-th slice (0 stops)."""
        self._check(self.lib.ftq_track_estimates(self.h, int(every)), "ftq_track_estimates")

    def slice_estimates(self):
        """The recorded slice estimates: dict(k, E, N (complex arrays), alive,
        E_avg, N_avg (complex): the averages over the recorded slices)."""
        import numpy as np
        cap = self.n_slices
        buf = (ctypes.c_double * (8 * (cap + 1)))()
        self._check(self.lib.ftq_slice_estimates(self.h, buf, cap), "ftq_slice_estimates")
        a = np.frombuffer(buf, dtype=np.float64).reshape(cap + 1, 8)
        n = int(a[0, 0])
        r = a[1:1 + n]
        return {"k": r[:, 0].astype(int), "E": r[:, 1] + 1j * r[:, 2], "N": r[:, 3] + 1j * r[:, 4],
                "alive": r[:, 5].astype(int), "E_avg": complex(a[0, 1], a[0, 2]),
                "N_avg": complex(a[0, 3], a[0, 4])}

    def set_green_kernel(self, kind):
        """Mixed path's G(tau) kernel: 0 by basis size, 1 tensor cores (Gauss-Jordan), 2 CUDA cores (LU)."""
        self._check(self.lib.ftq_set_green_kernel(self.h, int(kind)), "ftq_set_green_kernel")

    def set_wait_limit(self, polls):
        """Test hook: polls per mbarrier wait of the tensor-core kernels (-1: default)."""
        self._check(self.lib.ftq_set_wait_limit(self.h, int(polls)), "ftq_set_wait_limit")

    def status(self):
        v = ctypes.c_int()
        self._check(self.lib.ftq_status(self.h, ctypes.byref(v)), "ftq_status")
        return v.value


def _mu_estimates_impl():
    import torch

    class MuEstimates(torch.autograd.Function):
        """(<N>, <E>) at tau = beta of a whole path on fixed fields as a
        differentiable function of mu; the backward pass uses the library's
        mu derivative (fixed draws, frozen force bias)."""

        @staticmethod
        def forward(ctx, mu, system, fields, walkers, options):
            p = Propagator(system["N"], system["M"], system["rs"], system["theta"], system["dtau"],
                           mu=float(mu), walkers=walkers, **(options or {}))
            try:
                p.propagate(fields)
                g = p.mu_grad(per_walker=False)
            finally:
                p.close()
            ctx.save_for_backward(torch.tensor([g["dN"], g["dE"]], dtype=torch.float64))
            return torch.tensor([g["N"], g["E"]], dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad):
            (d,) = ctx.saved_tensors
            return (grad.to(torch.float64) * d).sum().reshape(()), None, None, None, None

    return MuEstimates


def mu_estimates(mu, system, fields, walkers, options=None):
    """torch wrapper: returns tensor([<N>, <E>]) differentiable in the 0-d tensor mu."""
    return _mu_estimates_impl().apply(mu, system, fields, walkers, options)


def tune_mu(system, fields, walkers, target_n, mu0, iterations=4, options=None):
    """Newton iteration mu <- mu - (<N> - N-bar) / (d<N>/dmu) on fixed fields
    (replaces the bracketing and least-squares fit of the paper's mu tuning)."""
    mu = float(mu0)
    history = []
    for _ in range(iterations):
        p = Propagator(system["N"], system["M"], system["rs"], system["theta"], system["dtau"], mu=mu,
                       walkers=walkers, **(options or {}))
        try:
            p.propagate(fields)
            g = p.mu_grad(per_walker=False)
        finally:
            p.close()
        history.append((mu, g["N"], g["dN"]))
        if g["dN"] == 0:
            break
        mu -= (g["N"] - target_n) / g["dN"]
    return mu, history


class Batch:
    """Ragged batch of UEG systems (ftq_init_batch), mixed precision.

    systems: list of dicts with N, M, rs, theta, dtau, walkers (mu optional)."""

    def __init__(self, systems, stabilise_every=5, exp_order=6, stream=None, seed=0):
        import torch
        if not torch.cuda.is_available():
            raise FTQError("no CUDA device: the batch has no CPU path")
        self._torch = torch
        self.lib = load_library()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr = (System * len(systems))()
        for k, sd in enumerate(systems):
            arr[k] = System(sd["N"], sd["M"], sd["rs"], sd["theta"], float(sd.get("mu", float("nan"))),
                            sd["dtau"], sd["walkers"], 0)
        o = Opts(0, stabilise_every, exp_order, FTQ_MIXED, FTQ_PHASELESS, 0, seed,
                 ctypes.c_void_p(self.stream.cuda_stream), 0.0)
        h = ctypes.c_void_p()
        st = self.lib.ftq_init_batch(ctypes.byref(h), len(systems), arr, ctypes.byref(o))
        if st != 0:
            raise FTQError(f"ftq_init_batch: {self.lib.ftq_last_error(None).decode()} (status {st})")
        self.h = h
        self.members = []
        for k, sd in enumerate(systems):
            mh = ctypes.c_void_p()
            if self.lib.ftq_batch_member(self.h, k, ctypes.byref(mh)) != 0:
                raise FTQError("ftq_batch_member failed")
            self.members.append(Propagator._member(self.lib, mh, sd["walkers"]))

    def propagate(self, fields):
        """fields: list of CUDA float64 tensors [n][W_s][N_alpha_s], same n for all."""
        t = self._torch
        n = int(fields[0].shape[0])
        ptrs = (ctypes.c_void_p * len(fields))()
        for k, (f, m) in enumerate(zip(fields, self.members)):
            if f.device.type != "cuda" or f.dtype != t.float64 or not f.is_contiguous():
                raise FTQError("fields must be contiguous CUDA float64 tensors")
            if f.shape[0] != n or f.shape[1] != m.W or f.shape[2] != m.n_alpha:
                raise FTQError(f"fields[{k}] must have shape [{n}, {m.W}, {m.n_alpha}]")
            ptrs[k] = f.data_ptr()
        st = self.lib.ftq_batch_propagate(self.h, n, ptrs)
        if st != 0:
            raise FTQError(f"ftq_batch_propagate: {self.lib.ftq_last_error(self.h).decode()} (status {st})")

    def autotune(self):
        n = len(self.members)
        ch = (ctypes.c_int * n)()
        ms = (ctypes.c_float * n)()
        st = self.lib.ftq_autotune(self.h, ch, ms)
        if st != 0:
            raise FTQError(f"ftq_autotune: {self.lib.ftq_last_error(self.h).decode()} (status {st})")
        return [(ch[k], ms[k]) for k in range(n)]

    def profile(self, enable=True):
        """Per-launch event timing of the batched launches (the graph is not
        used while a member is profiled)."""
        if self.lib.ftq_profile(self.h, 1 if enable else 0) != 0:
            raise FTQError("ftq_profile failed")

    def profile_read(self):
        """{kernel: (summed event ms, launches)} of the batched launches."""
        ms = (ctypes.c_double * K_COUNT)()
        n = (ctypes.c_int64 * K_COUNT)()
        if self.lib.ftq_profile_read(self.h, ms, n) != 0:
            raise FTQError("ftq_profile_read failed")
        return {k: (ms[v], n[v]) for k, v in KERNELS.items()}

    def launches(self):
        ms = (ctypes.c_double * K_COUNT)()
        total = 0
        for h in [self.h] + [m.h for m in self.members]:
            nn = (ctypes.c_int64 * K_COUNT)()
            self.lib.ftq_profile_read(h, ms, nn)
            total += sum(nn)
        return total

    def close(self):
        for m in self.members:
            m.h = None
        self.members = []
        if getattr(self, "h", None):
            self.lib.ftq_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
