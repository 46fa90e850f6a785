"""Python binding of the GB300 C-PCM / ISWIG library (libpcm.so).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI declared in include/pcm.h.  Arrays may be NumPy
arrays (host memory; the library copies them) or CUDA torch tensors (device
pointers, passed with PCM_PTR_DEVICE).  There is no CPU fallback: importing
this package fails if the compiled library is missing.

    from paper_1505_07851_gb300 import Context
    ctx = Context()
    M = ctx.build_surface(xyz, Z, radius)           # pcm_build_surface
    nbf = ctx.set_basis(atom, l, nprim, exps, coefs) # pcm_set_basis
    c = ctx.esp(P)                                   # pcm_esp
    q, st = ctx.solve(prev_diis_error=-1)            # pcm_solve
    dF = ctx.fock(q)                                 # pcm_fock
    E = ctx.energy(q)                                # pcm_energy
    g = ctx.gradient(q, P)                           # pcm_gradient

``SolvationEnergy`` wraps the whole path as a torch.autograd.Function of the
nuclear positions and the density: its backward is pcm_gradient (Eq. 14) for
the positions and pcm_fock (Eq. 10, the derivative of Eq. 13 with respect to
P) for the density.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "libpcm.so")

PCM_OK = 0
PCM_ERR_ARG = 1
PCM_ERR_CUDA = 2
PCM_ERR_OOM = 3
PCM_ERR_UNSUPPORTED = 4
PCM_ERR_NOT_CONVERGED = 5
PCM_ERR_TIMEOUT = 6
PCM_PTR_DEVICE = 1
PCM_ASYNC = 2
PCM_WARM = 4
PCM_GRAD_B = 8
PCM_GRAD_C = 16
PCM_GRAD_A = 32
PCM_TWO_DELTA = 64
PCM_APPLY_FP32 = 128
PCM_FP64 = 0
PCM_MIXED = 1
PRECOND = {"auto": 0, "none": 1, "jacobi": 2, "rbj": 3, "octree": 4}
OPERATOR = {"auto": 0, "stored": 1, "free": 2}   # pcm_options.operator_mode (PCM_MIXED)


class pcm_options(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("k", ctypes.c_double), ("zeta", ctypes.c_double),
                ("switch_drop", ctypes.c_double), ("schwarz", ctypes.c_double),
                ("rbj_block", ctypes.c_int), ("precond", ctypes.c_int), ("jacobi_below", ctypes.c_int),
                ("precision", ctypes.c_int), ("max_iter", ctypes.c_int), ("device", ctypes.c_int),
                ("seed", ctypes.c_ulonglong), ("stream", ctypes.c_void_p), ("timing", ctypes.c_int),
                ("autotune", ctypes.c_int), ("octree_leaf", ctypes.c_int), ("esp_variant", ctypes.c_int),
                ("fp32x2", ctypes.c_int), ("operator_mode", ctypes.c_int)]


class pcm_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("delta", ctypes.c_double),
                ("rnorm", ctypes.c_double), ("refinements", ctypes.c_int), ("M", ctypes.c_int),
                ("nbf", ctypes.c_int), ("pairs_candidate", ctypes.c_longlong),
                ("pairs_kept", ctypes.c_longlong), ("pairs_esp", ctypes.c_longlong),
                ("integrals_esp", ctypes.c_double), ("integrals_fock", ctypes.c_double),
                ("esp_class_pairs", ctypes.c_longlong * 6), ("fock_class_pairs", ctypes.c_longlong * 6),
                ("ms_esp_class", ctypes.c_double * 6), ("ms_fock_class", ctypes.c_double * 6),
                ("ms_solve", ctypes.c_double), ("ms_precond", ctypes.c_double), ("launches", ctypes.c_longlong),
                ("integrals_grad", ctypes.c_double), ("ms_grad", ctypes.c_double), ("operator_free", ctypes.c_int)]

    def as_dict(self):
        out = {}
        for f, _ in self._fields_:
            v = getattr(self, f)
            out[f] = list(v) if hasattr(v, "__len__") else v
        return out


class PCMError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__("%s failed: %s (%d)%s" % (where, _lib.pcm_strerror(status).decode(), status,
                                                   (": " + detail) if detail else ""))


def _load():
    if not os.path.exists(LIBPATH):
        raise ImportError("libpcm.so is not built (run __graft_entry__.build() or "
                          "python -m paper_1505_07851_gb300.build); there is no fallback")
    L = ctypes.CDLL(LIBPATH)
    vp = ctypes.c_void_p
    i = ctypes.c_int
    d = ctypes.c_double
    sig = {
        "pcm_default_options": (i, [ctypes.POINTER(pcm_options)]),
        "pcm_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(pcm_options)]),
        "pcm_destroy": (i, [vp]),
        "pcm_strerror": (ctypes.c_char_p, [i]),
        "pcm_last_error": (ctypes.c_char_p, []),
        "pcm_build_surface": (i, [vp, i, vp, vp, vp, i, ctypes.POINTER(i)]),
        "pcm_get_surface": (i, [vp, vp, vp, i]),
        "pcm_set_basis": (i, [vp, i, vp, vp, vp, vp, vp, ctypes.POINTER(i)]),
        "pcm_esp": (i, [vp, vp, vp, vp, i]),
        "pcm_solve": (i, [vp, vp, d, d, vp, ctypes.POINTER(pcm_stats), i]),
        "pcm_fock": (i, [vp, vp, vp, i]),
        "pcm_energy": (i, [vp, vp, vp, ctypes.POINTER(d), i]),
        "pcm_gradient": (i, [vp, vp, vp, vp, i]),
        "pcm_batch_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(pcm_options), i]),
        "pcm_batch_destroy": (i, [vp]),
        "pcm_batch_set_molecule": (i, [vp, i, i, vp, vp, vp, i, i, vp, vp, vp, vp, vp]),
        "pcm_batch_sizes": (i, [vp, i, ctypes.POINTER(i), ctypes.POINTER(i)]),
        "pcm_batch_run": (i, [vp, vp, d, vp, vp, vp, i]),
        "pcm_batch_get_stats": (i, [vp, i, ctypes.POINTER(pcm_stats)]),
        "pcm_get_stats": (i, [vp, ctypes.POINTER(pcm_stats)]),
        "pcm_autotune_table": (i, [vp, i]),
        "pcm_energy_noalloc": (i, [i, vp, i, vp, vp, vp, d, vp, vp]),
        "pcm_cg_threshold": (i, [d, d, i, ctypes.POINTER(d)]),
        "pcm_apply_a": (i, [vp, vp, vp, i]),
        "pcm_pipe_peak": (i, [i, i, ctypes.POINTER(d)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L, sorted(sig)


_lib, EXPORTS = _load()
globals().update({n: getattr(_lib, n) for n in EXPORTS})   # raw C entry points, same names


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype):
    """(pointer, flags, keepalive) for a NumPy array or a CUDA torch tensor."""
    if a is None:
        return None, 0, None
    if _is_torch(a):
        import torch
        want = torch.float64 if dtype == np.float64 else torch.int32
        if not a.is_cuda or a.dtype != want or not a.is_contiguous():
            raise TypeError("torch arguments must be contiguous CUDA tensors of dtype %s" % want)
        return a.data_ptr(), PCM_PTR_DEVICE, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, 0, arr


def cg_threshold(delta=-1.0, prev_diis_error=-1.0, two_delta=False):
    """The CG threshold pcm_solve uses (pcm_cg_threshold): fixed delta > 0,
    Eq. 21 from the previous DIIS error when delta <= 0, or the 2-delta
    scheme with two_delta=True.  Host logic; needs no GPU."""
    out = ctypes.c_double()
    st = _lib.pcm_cg_threshold(float(delta), float(prev_diis_error), PCM_TWO_DELTA if two_delta else 0,
                               ctypes.byref(out))
    if st != PCM_OK:
        raise PCMError(st, "pcm_cg_threshold", _lib.pcm_last_error().decode())
    return out.value


def pipe_peak(which="fp32", device=0):
    """Measured FMA throughput (TFLOP/s) of the "fp32", "fp64" or packed "fp32x2"
    pipe (pcm_pipe_peak)."""
    out = ctypes.c_double()
    st = _lib.pcm_pipe_peak(int(device), {"fp32": 0, "fp64": 1, "fp32x2": 2}[which], ctypes.byref(out))
    if st != PCM_OK:
        raise PCMError(st, "pcm_pipe_peak", _lib.pcm_last_error().decode())
    return out.value


def autotune_table():
    """The autotuner's choices so far: list of dicts (device, kernel, L,
    bucket, choice, fp32x2, trial_us) with kernel "esp_variant" (pair-driven
    with 4 or 2 points per thread, or MS-driven; "batch": the record of batch
    members, whose packed blocks run in one launch for all molecules) or
    "fock_pairs_per_thread" (1 or 2); trial_us the timed trial of each
    candidate in microseconds."""
    n = _lib.pcm_autotune_table(None, 0)
    buf = (ctypes.c_int * (8 * max(1, n)))()
    n = _lib.pcm_autotune_table(buf, n)
    names = {0: "pair-driven, 4 points/thread", 1: "pair-driven, 2 points/thread", 2: "MS-driven"}
    out = []
    for i in range(n):
        dev, kind, L, bucket, ch, t0, t1, t2 = buf[8 * i:8 * i + 8]
        packed = kind in (0, 1, 4)
        if kind in (0, 2, 4):
            trials = {names[v]: t for v, t in enumerate((t0, t1, t2)) if t > 0}
            out.append({"device": dev, "kernel": "esp_variant", "L": L, "bucket": bucket, "choice": names[ch],
                        "fp32x2": packed, "batch": kind == 4, "trial_us": trials})
        else:
            out.append({"device": dev, "kernel": "fock_pairs_per_thread", "L": L, "bucket": bucket, "choice": ch,
                        "fp32x2": packed, "trial_us": {1: t0, 2: t1}})
    return out


def energy_noalloc(A, Bz, c, q, f, E, stream=None):
    """pcm_energy_noalloc on CUDA torch tensors: A (M, >= M) row-major with
    unit column stride (its row stride is the leading dimension), Bz, c, q
    (M,), E (>= 1,) output, all float64 on one device; nothing is allocated
    by the library.  The call is made with that device current.  The result
    is ready once `stream` (default: torch's current stream of that device)
    reaches it."""
    import torch
    ts = (A, Bz, c, q, E)
    M = q.numel()
    if A.dim() != 2 or A.shape[0] < M or A.shape[1] < M or A.stride(1) != 1 or A.stride(0) < M:
        raise ValueError("energy_noalloc: A must be 2-D with at least (M, M) = (%d, %d) elements, unit column "
                         "stride and row stride >= M; got shape %s, strides %s" % (M, M, tuple(A.shape),
                                                                                   A.stride()))
    if Bz.numel() != M or c.numel() != M:
        raise ValueError("energy_noalloc: Bz and c must have M = %d elements (got %d, %d)"
                         % (M, Bz.numel(), c.numel()))
    if E.numel() < 1:
        raise ValueError("energy_noalloc: E must have at least one element")
    for t in ts:
        if not t.is_cuda or t.dtype != torch.float64:
            raise TypeError("energy_noalloc: arguments must be float64 CUDA tensors")
    for t in (Bz, c, q, E):
        if not t.is_contiguous():
            raise TypeError("energy_noalloc: Bz, c, q and E must be contiguous")
    if any(t.device != A.device for t in ts):
        raise ValueError("energy_noalloc: all tensors must be on one device (A is on %s)" % A.device)
    with torch.cuda.device(A.device):
        if stream is None:
            stream = torch.cuda.current_stream(A.device).cuda_stream
        st = _lib.pcm_energy_noalloc(M, A.data_ptr(), A.stride(0), Bz.data_ptr(), c.data_ptr(), q.data_ptr(),
                                     float(f), E.data_ptr(), stream)
    if st != PCM_OK:
        raise PCMError(st, "pcm_energy_noalloc", _lib.pcm_last_error().decode())
    return E


class Context:
    """One pcm_ctx: surface, basis, stored A and preconditioner on one GPU."""

    def __init__(self, eps=78.39, k=0.0, zeta=4.9, switch_drop=1e-8, schwarz=1e-12, rbj_block=100,
                 precond="auto", jacobi_below=1000, precision="fp64", max_iter=5000, device=0, seed=0,
                 stream=None, timing=False, autotune=False, octree_leaf=800, esp_variant=-1, fp32x2=True,
                 operator="auto"):
        o = pcm_options()
        _lib.pcm_default_options(ctypes.byref(o))
        o.eps, o.k, o.zeta, o.switch_drop, o.schwarz = eps, k, zeta, switch_drop, schwarz
        o.rbj_block, o.precond, o.jacobi_below = rbj_block, PRECOND[precond], jacobi_below
        o.precision = {"fp64": PCM_FP64, "mixed": PCM_MIXED}[precision]
        o.max_iter, o.device, o.seed = max_iter, device, seed
        o.stream = stream
        o.timing = 1 if timing else 0
        o.autotune = 1 if autotune else 0
        o.octree_leaf = int(octree_leaf)
        o.esp_variant = int(esp_variant)
        o.fp32x2 = 1 if fp32x2 else 0
        o.operator_mode = OPERATOR[operator]
        h = ctypes.c_void_p()
        self._check(_lib.pcm_create(ctypes.byref(h), ctypes.byref(o)), "pcm_create")
        self._h = h
        self.options = o
        self.M = 0
        self.nbf = 0
        self.natom = 0
        self.generation = 0          # incremented by every build_surface

    def _check(self, st, where, ok=(PCM_OK,)):
        if st not in ok:
            raise PCMError(st, where, _lib.pcm_last_error().decode())
        return st

    def close(self):
        if getattr(self, "_h", None):
            _lib.pcm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls -------------------------------------------------------------
    def build_surface(self, xyz, Z, radius, pts_per_sphere=110):
        xyz = np.ascontiguousarray(xyz, np.float64)
        Z = np.ascontiguousarray(Z, np.float64)
        radius = np.ascontiguousarray(radius, np.float64)
        M = ctypes.c_int()
        self._check(_lib.pcm_build_surface(self._h, len(Z), xyz.ctypes.data, Z.ctypes.data, radius.ctypes.data,
                                           int(pts_per_sphere), ctypes.byref(M)), "pcm_build_surface")
        self.M = M.value
        self.nbf = 0
        self.natom = len(Z)
        self.generation += 1
        return self.M

    def get_surface(self):
        xyzzs = np.zeros((self.M, 5))
        index = np.zeros(self.M, np.int32)
        self._check(_lib.pcm_get_surface(self._h, xyzzs.ctypes.data, index.ctypes.data, 0), "pcm_get_surface")
        return xyzzs, index

    def set_basis(self, shell_atom, shell_l, shell_nprim, exps, coefs):
        a = np.ascontiguousarray(shell_atom, np.int32)
        l = np.ascontiguousarray(shell_l, np.int32)
        n = np.ascontiguousarray(shell_nprim, np.int32)
        e = np.ascontiguousarray(exps, np.float64)
        c = np.ascontiguousarray(coefs, np.float64)
        nbf = ctypes.c_int()
        self._check(_lib.pcm_set_basis(self._h, len(l), a.ctypes.data, l.ctypes.data, n.ctypes.data,
                                       e.ctypes.data, c.ctypes.data, ctypes.byref(nbf)), "pcm_set_basis")
        self.nbf = nbf.value
        return self.nbf

    def _out(self, like, shape):
        if like is not None and _is_torch(like):
            import torch
            return torch.empty(shape, dtype=torch.float64, device=like.device)
        return np.zeros(shape)

    def esp(self, P, out=None, bz_out=None, async_=False):
        pP, fl, keep = _ptr(P, np.float64)
        c = out if out is not None else self._out(P, (self.M,))
        pc, flc, keepc = _ptr(c, np.float64)
        pb, flb, keepb = _ptr(bz_out, np.float64)
        if flc != fl or (bz_out is not None and flb != fl):
            raise TypeError("all array arguments must live on the same side (host or device)")
        flags = fl | (PCM_ASYNC if async_ else 0)
        self._check(_lib.pcm_esp(self._h, pP, pc, pb, flags), "pcm_esp")
        return c

    def solve(self, rhs=None, delta=-1.0, prev_diis_error=-1.0, q=None, warm=False, like=None, two_delta=False):
        """Returns (q, stats dict).  delta <= 0 selects the dynamic threshold of
        Eq. 21; two_delta=True makes delta the delta_2 of the 2-delta scheme
        (PCM_TWO_DELTA, Section 4b-i)."""
        pr, flr, keepr = _ptr(rhs, np.float64)
        if q is None:
            q = self._out(rhs if rhs is not None else like, (self.M,))
        pq, flq, keepq = _ptr(q, np.float64)
        if rhs is not None and flr != flq:
            raise TypeError("rhs and q must live on the same side (host or device)")
        st = pcm_stats()
        flags = flq | (PCM_WARM if warm else 0) | (PCM_TWO_DELTA if two_delta else 0)
        self._check(_lib.pcm_solve(self._h, pr, float(delta), float(prev_diis_error), pq, ctypes.byref(st),
                                   flags), "pcm_solve", ok=(PCM_OK, PCM_ERR_NOT_CONVERGED))
        return q, st.as_dict()

    def fock(self, q, out=None, async_=False):
        pq, fl, keep = _ptr(q, np.float64)
        dF = out if out is not None else self._out(q, (self.nbf, self.nbf))
        pF, flF, keepF = _ptr(dF, np.float64)
        if flF != fl:
            raise TypeError("q and dF must live on the same side (host or device)")
        self._check(_lib.pcm_fock(self._h, pq, pF, fl | (PCM_ASYNC if async_ else 0)), "pcm_fock")
        return dF

    def energy(self, q, c=None):
        pq, fl, keep = _ptr(q, np.float64)
        pc, flc, keepc = _ptr(c, np.float64)
        if c is not None and flc != fl:
            raise TypeError("q and c must live on the same side (host or device)")
        E = ctypes.c_double()
        self._check(_lib.pcm_energy(self._h, pq, pc, ctypes.byref(E), fl), "pcm_energy")
        return E.value

    def apply_a(self, x, out=None, fp32=False):
        """y = A x (pcm_apply_a): the solver's accurate product, or with fp32
        the FP32 matrix-free product of the inner PCM_MIXED solver."""
        px, fl, keep = _ptr(x, np.float64)
        y = out if out is not None else self._out(x, (self.M,))
        py, fly, keepy = _ptr(y, np.float64)
        if fly != fl:
            raise TypeError("x and y must live on the same side (host or device)")
        self._check(_lib.pcm_apply_a(self._h, px, py, fl | (PCM_APPLY_FP32 if fp32 else 0)), "pcm_apply_a")
        return y

    def gradient(self, q, P=None, out=None, terms="BCA", async_=False):
        """Nuclear gradient (natom, 3) of Eq. 13 at fixed P and q (Eq. 14):
        terms is any combination of "B" (z^T dB q), "C" (the integrals, needs
        P) and "A" (q^T dA q / 2f, with the switching factors)."""
        pq, fl, keep = _ptr(q, np.float64)
        pP, flP, keepP = _ptr(P, np.float64)
        g = out if out is not None else self._out(q, (self.natom, 3))
        pg, flg, keepg = _ptr(g, np.float64)
        if flg != fl or (P is not None and flP != fl):
            raise TypeError("q, P and the output must live on the same side (host or device)")
        bits = {"B": PCM_GRAD_B, "C": PCM_GRAD_C, "A": PCM_GRAD_A}
        flags = fl | (PCM_ASYNC if async_ else 0)
        for t in terms:
            flags |= bits[t]
        self._check(_lib.pcm_gradient(self._h, pP, pq, pg, flags), "pcm_gradient")
        return g

    def stats(self):
        st = pcm_stats()
        self._check(_lib.pcm_get_stats(self._h, ctypes.byref(st)), "pcm_get_stats")
        return st.as_dict()

    # -- convenience -------------------------------------------------------
    def setup(self, mol, basis, pts_per_sphere=110):
        """build_surface + set_basis from workload-style objects."""
        M = self.build_surface(mol.xyz, mol.Z, mol.radius, pts_per_sphere)
        nbf = self.set_basis(basis.shell_atom, basis.shell_l, basis.shell_nprim, basis.exps, basis.coefs)
        return M, nbf



class Batch:
    """One pcm_batch: many molecules run together (pcm_batch_run)."""

    def __init__(self, nmol, eps=78.39, k=0.0, zeta=4.9, switch_drop=1e-8, schwarz=1e-12, rbj_block=100,
                 precond="auto", jacobi_below=1000, precision="mixed", max_iter=5000, device=0, seed=0,
                 stream=None, autotune=True, fp32x2=True, operator="auto"):
        o = pcm_options()
        _lib.pcm_default_options(ctypes.byref(o))
        o.eps, o.k, o.zeta, o.switch_drop, o.schwarz = eps, k, zeta, switch_drop, schwarz
        o.rbj_block, o.precond, o.jacobi_below = rbj_block, PRECOND[precond], jacobi_below
        o.precision = {"fp64": PCM_FP64, "mixed": PCM_MIXED}[precision]
        o.max_iter, o.device, o.seed, o.stream = max_iter, device, seed, stream
        o.autotune = 1 if autotune else 0
        o.fp32x2 = 1 if fp32x2 else 0
        o.operator_mode = OPERATOR[operator]
        h = ctypes.c_void_p()
        st = _lib.pcm_batch_create(ctypes.byref(h), ctypes.byref(o), int(nmol))
        if st != PCM_OK:
            raise PCMError(st, "pcm_batch_create", _lib.pcm_last_error().decode())
        self._h = h
        self.nmol = int(nmol)
        self.device = device
        self.sizes = [None] * self.nmol

    def _check(self, st, where):
        if st != PCM_OK:
            raise PCMError(st, where, _lib.pcm_last_error().decode())

    def close(self):
        if getattr(self, "_h", None):
            _lib.pcm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_molecule(self, i, mol, basis, pts_per_sphere=110):
        xyz = np.ascontiguousarray(mol.xyz, np.float64)
        Z = np.ascontiguousarray(mol.Z, np.float64)
        rad = np.ascontiguousarray(mol.radius, np.float64)
        a = np.ascontiguousarray(basis.shell_atom, np.int32)
        l = np.ascontiguousarray(basis.shell_l, np.int32)
        n = np.ascontiguousarray(basis.shell_nprim, np.int32)
        e = np.ascontiguousarray(basis.exps, np.float64)
        c = np.ascontiguousarray(basis.coefs, np.float64)
        self._check(_lib.pcm_batch_set_molecule(self._h, int(i), len(Z), xyz.ctypes.data, Z.ctypes.data,
                                                rad.ctypes.data, int(pts_per_sphere), len(l), a.ctypes.data,
                                                l.ctypes.data, n.ctypes.data, e.ctypes.data, c.ctypes.data),
                    "pcm_batch_set_molecule")
        M, nbf = ctypes.c_int(), ctypes.c_int()
        self._check(_lib.pcm_batch_sizes(self._h, int(i), ctypes.byref(M), ctypes.byref(nbf)), "pcm_batch_sizes")
        self.sizes[i] = (M.value, nbf.value)
        return self.sizes[i]

    def run(self, Ps, delta, want_q=False, want_dF=False, dF_out=None):
        """Ps: nmol densities (all NumPy arrays or all CUDA tensors).  Returns
        (E, q list or None, dF list or None); outputs live where Ps live.
        dF_out: caller-owned Fock-correction outputs (one per molecule)."""
        if len(Ps) != self.nmol:
            raise ValueError("one density per molecule")
        dev = _is_torch(Ps[0])
        keep = []
        P_ptrs = (ctypes.c_void_p * self.nmol)()
        for i, P in enumerate(Ps):
            p, fl, k = _ptr(P, np.float64)
            if bool(fl) != dev:
                raise TypeError("all densities must live on the same side (host or device)")
            P_ptrs[i] = p
            keep.append(k)
        E = np.zeros(self.nmol)
        q = dF = None
        q_ptrs = dF_ptrs = None
        if want_q:
            q = [self._alloc(Ps[i], (self.sizes[i][0],)) for i in range(self.nmol)]
            q_ptrs = (ctypes.c_void_p * self.nmol)(*[_ptr(a, np.float64)[0] for a in q])
        if want_dF or dF_out is not None:
            dF = list(dF_out) if dF_out is not None else \
                [self._alloc(Ps[i], (self.sizes[i][1], self.sizes[i][1])) for i in range(self.nmol)]
            for i, a in enumerate(dF):
                if tuple(a.shape) != (self.sizes[i][1], self.sizes[i][1]) or _is_torch(a) != dev:
                    raise TypeError("dF_out[%d] must be an nbf x nbf array on the densities' side" % i)
            dF_ptrs = (ctypes.c_void_p * self.nmol)(*[_ptr(a, np.float64)[0] for a in dF])
        self._check(_lib.pcm_batch_run(self._h, P_ptrs, float(delta), E.ctypes.data, q_ptrs, dF_ptrs,
                                       PCM_PTR_DEVICE if dev else 0), "pcm_batch_run")
        return E, q, dF

    def _alloc(self, like, shape):
        if _is_torch(like):
            import torch
            return torch.empty(shape, dtype=torch.float64, device=like.device)
        return np.zeros(shape)

    def stats(self, i=-1):
        st = pcm_stats()
        self._check(_lib.pcm_batch_get_stats(self._h, int(i), ctypes.byref(st)), "pcm_batch_get_stats")
        return st.as_dict()


# --------------------------------------------------------------------------
# autograd
# --------------------------------------------------------------------------
def _autograd_function():
    import torch

    class SolvationEnergy(torch.autograd.Function):
        """Delta G_els (Eq. 13) as a function of the nuclear positions xyz
        (natom, 3) and the density P (nbf, nbf, CUDA float64), with q solved
        from Eq. 1 to `delta` in the forward pass.  Backward: dG/dxyz by
        pcm_gradient (Eq. 14; exact at the solution of Eq. 1 because Eq. 13 is
        stationary in q) and dG/dP = dF by pcm_fock (Eq. 10)."""

        @staticmethod
        def forward(fctx, xyz, P, pcm, mol, basis, delta):
            x = xyz.detach().to("cpu", torch.float64).numpy()
            pcm.build_surface(x, mol.Z, mol.radius)
            pcm.set_basis(basis.shell_atom, basis.shell_l, basis.shell_nprim, basis.exps, basis.coefs)
            Pd = P.detach().contiguous()
            pcm.esp(Pd)
            q, _ = pcm.solve(delta=delta, like=Pd)
            E = pcm.energy(q)
            fctx.save_for_backward(Pd, q)
            fctx.pcm, fctx.mol, fctx.basis = pcm, mol, basis
            fctx.generation = pcm.generation
            fctx.x = x
            fctx.xyz_device = xyz.device
            return torch.tensor(E, dtype=torch.float64, device=P.device)

        @staticmethod
        def backward(fctx, gE):
            Pd, q = fctx.saved_tensors
            pcm = fctx.pcm
            if pcm.generation != fctx.generation:        # the context moved on: rebuild this geometry
                b = fctx.basis
                pcm.build_surface(fctx.x, fctx.mol.Z, fctx.mol.radius)
                pcm.set_basis(b.shell_atom, b.shell_l, b.shell_nprim, b.exps, b.coefs)
                fctx.generation = pcm.generation
            gx = gP = None
            if fctx.needs_input_grad[0]:
                gx = (gE * pcm.gradient(q, Pd)).to(fctx.xyz_device)
            if fctx.needs_input_grad[1]:
                gP = gE * pcm.fock(q)
            return gx, gP, None, None, None, None

    return SolvationEnergy


def solvation_energy(xyz, P, pcm, mol, basis, delta=1e-10):
    """Differentiable Delta G_els(xyz, P) on the context `pcm` (see
    SolvationEnergy); mol supplies Z and the cavity radii, basis the shells."""
    global SolvationEnergy
    if SolvationEnergy is None:
        SolvationEnergy = _autograd_function()
    return SolvationEnergy.apply(xyz, P, pcm, mol, basis, float(delta))


SolvationEnergy = None
