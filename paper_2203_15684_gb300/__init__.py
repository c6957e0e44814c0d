"""Python binding of the GB300 DFPT Hubbard-parameter engine (C ABI in include/hp.h).

Argument marshalling only: every step of the computation runs in the CUDA kernels of
``libhpgb.so``.  There is no CPU fallback; if the library is missing the import of a function
raises, and a call on a machine without a GPU returns HP_ECUDA.

    ctx = Context.from_workload(w)          # hp_setup
    ctx.ground_state(nelec, nspin, moments) # hp_ground_state  (or ctx.set_ground_state(...))
    dn0, dn, info = ctx.response(iq, atom)  # hp_response
    chi0, chi, hub = ctx.hubbard()          # hp_hubbard
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhpgb.so")

STATUS = {0: "HP_OK", 1: "HP_EINVAL", 2: "HP_ENOMEM", 3: "HP_ESTATE", 4: "HP_ENOTCONV", 5: "HP_ENUMERIC",
          6: "HP_ECUDA", 7: "HP_ETIMEOUT", 8: "HP_ESINGULAR", 9: "HP_ENOGAP", 10: "HP_ENOTIMPL"}
HP_OK, HP_ENOTCONV = 0, 4


class HPError(RuntimeError):
    def __init__(self, code, where, msg=""):
        self.code = code
        super().__init__("%s failed: %s %s" % (where, STATUS.get(code, code), msg))


class Species(C.Structure):
    _fields_ = [("amp", C.c_double), ("width", C.c_double), ("l_proj", C.c_int), ("D", C.c_double),
                ("proj_width", C.c_double), ("l_hub", C.c_int), ("hub_width", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("cg_tol", C.c_double), ("cg_maxiter", C.c_int), ("scf_tol", C.c_double),
                ("conv_thr_chi", C.c_double), ("niter_max", C.c_int), ("nmix", C.c_int), ("alpha_mix", C.c_double),
                ("gs_tol", C.c_double), ("gs_maxiter", C.c_int), ("fft_grid", C.c_int * 3), ("band_batch", C.c_int),
                ("cuda_stream", C.c_void_p), ("cg_adapt", C.c_double), ("mixed_floor", C.c_double),
                ("wait_timeout_s", C.c_double), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
                ("alloc_user", C.c_void_p), ("hub_ortho", C.c_int)]


class Sizes(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("nk", "nq", "nspin", "nocc", "nbnd")] + [("grid", C.c_int * 3), ("nr", C.c_int)] + \
               [(n, C.c_int) for n in ("nat", "nhub_atoms", "nhub_orb", "nproj", "mmax", "npw_max", "ncell", "nchi")]


class GsInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("residual", C.c_double), ("gap", C.c_double), ("homo", C.c_double),
                ("lumo", C.c_double), ("seconds", C.c_double)]


class RespInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("cg_iterations", C.c_longlong), ("hpsi", C.c_longlong),
                ("residual", C.c_double), ("dchi", C.c_double), ("seconds", C.c_double), ("stagnated", C.c_int)]


class PairV(C.Structure):
    _fields_ = [("s", C.c_int), ("jchi", C.c_int), ("dist", C.c_double), ("V", C.c_double), ("j", C.c_int),
                ("R", C.c_int * 3)]


class KernelStats(C.Structure):
    _fields_ = [("ms", C.c_double), ("launches", C.c_longlong), ("flops", C.c_double), ("bytes", C.c_double)]


# kernel families timed by profile_begin/profile_end, in the order of HP_KF_*
KERNEL_FAMILIES = ("fft_pass", "column", "plane", "project", "expand")

_lib = None

SYMBOLS = ["hp_default_options", "hp_setup", "hp_query_sizes", "hp_sphere", "hp_hubbard_atoms", "hp_ground_state",
           "hp_set_ground_state", "hp_get_ground_state", "hp_apply_h", "hp_response", "hp_hubbard", "hp_last_error",
           "hp_destroy", "hp_selftest_fft_host", "hp_selftest_eigh", "hp_get_wavefunctions", "hp_profile_begin",
           "hp_profile_end", "hp_launch_count", "hp_apply_h_noalloc", "hp_set_precision", "hp_selftest_convert",
           "hp_batch_run", "hp_alloc_count", "hp_sphere_kq", "hp_apply_sternheimer", "hp_selftest_xc",
           "hp_selftest_tc", "hp_set_hubbard", "hp_bare_levels", "hp_perturbed_atoms", "hp_irreducible_q",
           "hp_irreducible_pairs"]


def lib():
    """The loaded engine library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libhpgb.so is not built (run `python -m paper_2203_15684_gb300.build`); "
                           "there is no CPU fallback")
    L = C.CDLL(LIB_PATH)
    P, I, D, V = C.POINTER, C.c_int, C.c_double, C.c_void_p
    L.hp_default_options.argtypes = [P(Options)]
    L.hp_default_options.restype = None
    L.hp_setup.argtypes = [P(D), I, P(Species), I, P(I), P(D), D, P(I), P(I), P(Options), P(V)]
    L.hp_query_sizes.argtypes = [V, P(Sizes)]
    L.hp_sphere.argtypes = [V, I, P(I), P(I)]
    L.hp_hubbard_atoms.argtypes = [V, P(I), P(I)]
    L.hp_ground_state.argtypes = [V, D, I, P(I), D, P(GsInfo)]
    L.hp_set_ground_state.argtypes = [V, I, D, P(D), P(D), P(D), P(D)]
    L.hp_get_ground_state.argtypes = [V, P(D), P(D), P(D)]
    L.hp_apply_h.argtypes = [V, I, I, I, P(D), P(D)]
    L.hp_response.argtypes = [V, I, I, P(D), P(D), P(RespInfo)]
    L.hp_hubbard.argtypes = [V, P(D), P(D), P(D), P(D), P(PairV), P(I)]
    L.hp_last_error.argtypes = [V]
    L.hp_last_error.restype = C.c_char_p
    L.hp_destroy.argtypes = [V]
    L.hp_destroy.restype = None
    L.hp_selftest_fft_host.argtypes = [I, I, I, P(D), P(D)]
    L.hp_selftest_eigh.argtypes = [I, I, P(D), P(D), P(D)]
    L.hp_get_wavefunctions.argtypes = [V, P(D)]
    L.hp_profile_begin.argtypes = []
    L.hp_profile_begin.restype = None
    L.hp_profile_end.argtypes = [P(KernelStats)]
    L.hp_launch_count.argtypes = []
    L.hp_apply_h_noalloc.argtypes = [V, I, I, I, V, V, V]
    L.hp_set_precision.argtypes = [V, I]
    L.hp_selftest_convert.argtypes = [C.c_longlong, P(D), P(C.c_float), P(D), P(C.c_float), P(D)]
    L.hp_batch_run.argtypes = [I, P(V), P(P(D)), P(P(D)), P(P(D)), P(I)]
    L.hp_alloc_count.argtypes = []
    L.hp_sphere_kq.argtypes = [V, I, I, P(I), P(I)]
    L.hp_apply_sternheimer.argtypes = [V, I, I, I, I, P(D), P(D), P(D)]
    L.hp_selftest_xc.argtypes = [I, I, P(D), P(D), P(D)]
    L.hp_selftest_tc.argtypes = [I, I, I, P(C.c_float), P(C.c_float), P(C.c_float), I, D]
    L.hp_set_hubbard.argtypes = [V, P(D), I, P(PairV)]
    L.hp_bare_levels.argtypes = [V, I, I, P(D)]
    L.hp_perturbed_atoms.argtypes = [V, I, D, D, P(I), P(I), P(I), P(D)]
    L.hp_irreducible_q.argtypes = [V, P(I), P(I), P(I)]
    L.hp_irreducible_pairs.argtypes = [V, P(I), P(I), P(I)]
    for n in SYMBOLS:
        f = getattr(L, n)
        if n in ("hp_launch_count", "hp_alloc_count"):
            f.restype = C.c_longlong
        elif n not in ("hp_default_options", "hp_last_error", "hp_destroy", "hp_profile_begin"):
            f.restype = I
    _lib = L
    return L


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def default_options(**kw):
    o = Options()
    lib().hp_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "fft_grid":
            for i in range(3):
                o.fft_grid[i] = int(v[i]) if v is not None else 0
        else:
            setattr(o, k, v)
    return o


def selftest_fft_host(x, sign):
    """Runs the engine's Stockham stage code on the host: x (nlines, n) complex."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    nlines, n = x.shape
    out = np.empty_like(x)
    st = lib().hp_selftest_fft_host(n, nlines, sign, _dptr(x.view(np.float64)), _dptr(out.view(np.float64)))
    if st != HP_OK:
        raise HPError(st, "hp_selftest_fft_host")
    return out


def selftest_eigh(A):
    """Batched Hermitian eigensolver of the ground state on the GPU: A (nbatch, n, n) complex."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    nb, n, _ = A.shape
    w = np.zeros((nb, n))
    V = np.zeros_like(A)
    st = lib().hp_selftest_eigh(n, nb, _dptr(A.view(np.float64)), _dptr(w), _dptr(V.view(np.float64)))
    if st != HP_OK:
        raise HPError(st, "hp_selftest_eigh")
    return w, V


def selftest_convert(x):
    """-> (f, back, f_ref, back_ref): the library's integer-operation FP64 -> FP32 -> FP64
    conversions of the float64 array x and the hardware conversions, computed on the GPU."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.size
    f, fr = np.zeros(n, np.float32), np.zeros(n, np.float32)
    b, br = np.zeros(n), np.zeros(n)
    fp = lambda a: a.ctypes.data_as(C.POINTER(C.c_float))
    st = lib().hp_selftest_convert(n, _dptr(x), fp(f), _dptr(b), fp(fr), _dptr(br))
    if st != HP_OK:
        raise HPError(st, "hp_selftest_convert")
    return f, b, fr, br


def profile_begin():
    lib().hp_profile_begin()


def profile_end():
    """-> {family: dict(ms, launches, flops, bytes)} for the kernel families timed since
    profile_begin() (names in KERNEL_FAMILIES)."""
    stats = (KernelStats * len(KERNEL_FAMILIES))()
    st = lib().hp_profile_end(stats)
    if st != HP_OK:
        raise HPError(st, "hp_profile_end")
    return {name: dict(ms=x.ms, launches=x.launches, flops=x.flops, bytes=x.bytes)
            for name, x in zip(KERNEL_FAMILIES, stats)}


def launch_count():
    return int(lib().hp_launch_count())


def alloc_count():
    """Device allocations the library has made in this process."""
    return int(lib().hp_alloc_count())


def selftest_xc(rho):
    """LDA potential and kernel of the library on the GPU: rho (nspin, n) -> (vxc (nspin, n),
    fxc (1 or 3, n))."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    nspin, n = rho.shape
    v = np.zeros_like(rho)
    f = np.zeros((1 if nspin == 1 else 3, n))
    st = lib().hp_selftest_xc(n, nspin, _dptr(rho), _dptr(v), _dptr(f))
    if st != HP_OK:
        raise HPError(st, "hp_selftest_xc")
    return v, f


def selftest_tc(A, B, lbo_swap=0, timeout_s=2.0, four=False, drain=False):
    """D = A B^T on the tensor cores (tcgen05 kind::tf32, three-product TF32 split; four: also a_lo b_lo;
    drain: accumulator drained to FP64 every 32 values of K): A (M, K), B (N, K) float32 -> D (M, N)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    M, K = A.shape
    N = B.shape[0]
    D = np.zeros((M, N), dtype=np.float32)
    fp = lambda a: a.ctypes.data_as(C.POINTER(C.c_float))
    mode = (1 if lbo_swap else 0) | (2 if four else 0) | (4 if drain else 0)
    st = lib().hp_selftest_tc(M, N, K, fp(A), fp(B), fp(D), mode, float(timeout_s))
    if st != HP_OK:
        raise HPError(st, "hp_selftest_tc")
    return D


class TorchAllocator:
    """dev_alloc / dev_free callbacks that take the library's device buffers from PyTorch's caching
    allocator on a given CUDA stream (argument marshalling only; the library decides what to
    allocate)."""

    def __init__(self, stream=None, device=None):
        import torch

        self._torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self.stream = stream
        self.alloc_fn = ALLOC_FN(self._alloc)
        self.free_fn = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            return int(self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
        except Exception:
            return None

    def _free(self, ptr, user):
        try:
            self._torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass


class Context:
    """An hp_ctx: one crystal, its ground state and its response columns."""

    def __init__(self, cell, species, atoms, ecutwfc, kmesh, qmesh, options=None, torch_alloc=None):
        """torch_alloc: take device memory from PyTorch's caching allocator (on the options' CUDA
        stream); None = whenever torch sees a GPU."""
        L = lib()
        self._ptr = C.c_void_p()
        self._alloc = None
        cell = np.ascontiguousarray(np.asarray(cell, dtype=np.float64).reshape(9))
        sp = (Species * len(species))()
        for i, s in enumerate(species):
            sp[i] = Species(s["amp"], s["width"], int(s["l_proj"]), s["D"], s["proj_width"], int(s["l_hub"]),
                            s["hub_width"])
        kinds = np.ascontiguousarray([int(a[0]) for a in atoms], dtype=np.int32)
        frac = np.ascontiguousarray([list(a[1]) for a in atoms], dtype=np.float64).reshape(-1)
        km = np.ascontiguousarray(kmesh, dtype=np.int32)
        qm = np.ascontiguousarray(qmesh, dtype=np.int32)
        opt = options if options is not None else default_options()
        if torch_alloc is None:
            try:
                import torch

                torch_alloc = torch.cuda.is_available()
            except ImportError:
                torch_alloc = False
        if torch_alloc:
            self._alloc = TorchAllocator(stream=opt.cuda_stream or 0)
            opt.dev_alloc = self._alloc.alloc_fn
            opt.dev_free = self._alloc.free_fn
        st = L.hp_setup(_dptr(cell), len(species), sp, len(kinds), _iptr(kinds), _dptr(frac), float(ecutwfc),
                        _iptr(km), _iptr(qm), C.byref(opt), C.byref(self._ptr))
        if st != HP_OK:
            raise HPError(st, "hp_setup")

    @classmethod
    def from_workload(cls, w, torch_alloc=None, **opts):
        opts.setdefault("fft_grid", w.get("grid"))
        opts.setdefault("hub_ortho", 1 if w.get("hubbard_projectors", "atomic") == "ortho-atomic" else 0)
        return cls(w["cell"], w["species"], w["atoms"], w["ecutwfc"], w["kmesh"], w["qmesh"], default_options(**opts),
                   torch_alloc=torch_alloc)

    # -------------------------------------------------------------------------------------------
    def _check(self, st, where, ok=(HP_OK,)):
        if st not in ok:
            raise HPError(st, where, self.last_error())
        return st

    def last_error(self):
        return lib().hp_last_error(self._ptr).decode()

    def destroy(self):
        if self._ptr:
            import sys

            # at interpreter exit PyTorch may already be gone: leave the buffers to the process exit
            if not (self._alloc is not None and sys.is_finalizing()):
                lib().hp_destroy(self._ptr)
            self._ptr = C.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def set_precision(self, precision):
        """0 = FP64, 1 = mixed (FP32 grids and projections, FP64 vectors and scalars)."""
        self._check(lib().hp_set_precision(self._ptr, int(precision)), "hp_set_precision")

    def query_sizes(self):
        s = Sizes()
        self._check(lib().hp_query_sizes(self._ptr, C.byref(s)), "hp_query_sizes")
        d = {n: getattr(s, n) for n, _ in Sizes._fields_}
        d["grid"] = tuple(s.grid)
        return d

    def sphere(self, ik):
        n = C.c_int()
        self._check(lib().hp_sphere(self._ptr, ik, C.byref(n), None), "hp_sphere")
        m = np.zeros((n.value, 3), dtype=np.int32)
        self._check(lib().hp_sphere(self._ptr, ik, C.byref(n), _iptr(m)), "hp_sphere")
        return m

    def hubbard_atoms(self):
        nh = self.query_sizes()["nhub_atoms"]
        a = np.zeros(nh, dtype=np.int32)
        m = np.zeros(nh, dtype=np.int32)
        self._check(lib().hp_hubbard_atoms(self._ptr, _iptr(a), _iptr(m)), "hp_hubbard_atoms")
        return a, m

    def ground_state(self, nelec, nspin, moments=None, tot_mag=0.0):
        info = GsInfo()
        mom = None
        if moments is not None:
            mom_a = np.ascontiguousarray(moments, dtype=np.int32)
            mom = _iptr(mom_a)
        st = lib().hp_ground_state(self._ptr, float(nelec), int(nspin), mom, float(tot_mag), C.byref(info))
        self._check(st, "hp_ground_state")
        return {n: getattr(info, n) for n, _ in GsInfo._fields_}

    def set_ground_state(self, nspin, nelec, vhxc, rho, eps, psi):
        """psi: list over spin of lists over k of (npw_k, nocc) complex arrays in sphere order."""
        vh = np.ascontiguousarray(vhxc, dtype=np.float64).reshape(-1)
        rh = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        ep = np.ascontiguousarray(eps, dtype=np.float64).reshape(-1)
        flat = np.concatenate([np.ascontiguousarray(psi[s][k].T).reshape(-1) for s in range(nspin)
                               for k in range(len(psi[s]))]).astype(np.complex128)
        self._check(lib().hp_set_ground_state(self._ptr, int(nspin), float(nelec), _dptr(vh), _dptr(rh), _dptr(ep),
                                              _dptr(flat.view(np.float64))), "hp_set_ground_state")

    def get_ground_state(self):
        s = self.query_sizes()
        eps = np.zeros((s["nspin"], s["nk"], s["nocc"]))
        rho = np.zeros((s["nspin"], s["nr"]))
        vhxc = np.zeros((s["nspin"], s["nr"]))
        self._check(lib().hp_get_ground_state(self._ptr, _dptr(eps), _dptr(rho), _dptr(vhxc)), "hp_get_ground_state")
        return eps, rho, vhxc

    def get_wavefunctions(self):
        """Packed occupied wavefunctions (complex), the layout set_ground_state reads."""
        s = self.query_sizes()
        n = sum(len(self.sphere(k)) for k in range(s["nk"])) * s["nocc"] * s["nspin"]
        out = np.zeros(n, dtype=np.complex128)
        self._check(lib().hp_get_wavefunctions(self._ptr, _dptr(out.view(np.float64))), "hp_get_wavefunctions")
        return out

    def set_ground_state_packed(self, nspin, nelec, vhxc, rho, eps, psi_packed):
        vh = np.ascontiguousarray(vhxc, dtype=np.float64).reshape(-1)
        rh = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        ep = np.ascontiguousarray(eps, dtype=np.float64).reshape(-1)
        ps = np.ascontiguousarray(psi_packed, dtype=np.complex128)
        self._check(lib().hp_set_ground_state(self._ptr, int(nspin), float(nelec), _dptr(vh), _dptr(rh), _dptr(ep),
                                              _dptr(ps.view(np.float64))), "hp_set_ground_state")

    def apply_h(self, ik, spin, psi):
        """psi: (nb, npw_k) complex in sphere order -> H psi, same shape."""
        x = np.ascontiguousarray(psi, dtype=np.complex128)
        out = np.empty_like(x)
        self._check(lib().hp_apply_h(self._ptr, ik, spin, x.shape[0], _dptr(x.view(np.float64)),
                                     _dptr(out.view(np.float64))), "hp_apply_h")
        return out

    def apply_h_noalloc(self, ik, spin, nb, psi_dev_ptr, out_dev_ptr, stream=None):
        """H psi on caller-owned device rows (nb x npw_max complex); allocates nothing."""
        st = lib().hp_apply_h_noalloc(self._ptr, int(ik), int(spin), int(nb), C.c_void_p(psi_dev_ptr),
                                      C.c_void_p(out_dev_ptr), C.c_void_p(stream) if stream else None)
        self._check(st, "hp_apply_h_noalloc")

    def response(self, iq, atom):
        """Returns (dn0, dn, info); dn arrays complex [nhub_atoms][nspin][mmax][mmax]."""
        s = self.query_sizes()
        shape = (s["nhub_atoms"], s["nspin"], s["mmax"], s["mmax"])
        dn0 = np.zeros(shape, dtype=np.complex128)
        dn = np.zeros(shape, dtype=np.complex128)
        info = RespInfo()
        st = lib().hp_response(self._ptr, int(iq), int(atom), _dptr(dn0.view(np.float64)), _dptr(dn.view(np.float64)),
                               C.byref(info))
        self._check(st, "hp_response")
        return dn0, dn, {n: getattr(info, n) for n, _ in RespInfo._fields_}

    def hubbard(self):
        """-> (chi0, chi, hub): the supercell response matrices and (chi0^-1 - chi^-1) in eV."""
        r = self.hubbard_parameters()
        return r["chi0"], r["chi"], r["hub"]

    def hubbard_parameters(self):
        """-> dict(chi0, chi, hub, U (eV per Hubbard atom), V: list of (s, jchi, dist_bohr, V_eV))."""
        s = self.query_sizes()
        n, nh = s["nchi"], s["nhub_atoms"]
        chi0, chi, hub, U = np.zeros((n, n)), np.zeros((n, n)), np.zeros((n, n)), np.zeros(nh)
        cap = C.c_int(0)
        self._check(lib().hp_hubbard(self._ptr, _dptr(chi0), _dptr(chi), _dptr(hub), _dptr(U), None, C.byref(cap)),
                    "hp_hubbard")
        pairs = (PairV * max(1, cap.value))()
        self._check(lib().hp_hubbard(self._ptr, None, None, None, None, pairs, C.byref(cap)), "hp_hubbard")
        V = [(p.s, p.jchi, p.dist, p.V) for p in pairs[: cap.value]]
        Vpairs = [(p.s, p.j, tuple(p.R), p.V) for p in pairs[: cap.value]]
        return dict(chi0=chi0, chi=chi, hub=hub, U=U, V=V, pairs=Vpairs)

    def set_hubbard(self, U=None, pairs=()):
        """DFT+U+V ground state (hp_set_hubbard): U (eV per Hubbard atom, or None) and pairs
        [(s, j, (R1, R2, R3), V_eV)] of Hubbard-atom indices, as hubbard_parameters()["pairs"]."""
        nh = self.query_sizes()["nhub_atoms"]
        u = None
        if U is not None:
            u_a = np.ascontiguousarray(U, dtype=np.float64).reshape(nh)
            u = _dptr(u_a)
        arr = (PairV * max(1, len(pairs)))()
        for i, (s_, j, R, v) in enumerate(pairs):
            arr[i].s, arr[i].j, arr[i].V = int(s_), int(j), float(v)
            for d in range(3):
                arr[i].R[d] = int(R[d])
        self._check(lib().hp_set_hubbard(self._ptr, u, len(pairs), arr), "hp_set_hubbard")

    def bare_levels(self, nlev, ik=0):
        """Lowest nlev eigenvalues of T + V_loc + V_NL at mesh point ik (hp_bare_levels)."""
        e = np.zeros(int(nlev))
        self._check(lib().hp_bare_levels(self._ptr, int(ik), int(nlev), _dptr(e)), "hp_bare_levels")
        return e

    def perturbed_atoms(self, find_atpert=1, docc_thr=5e-5, dist_thr=6e-4):
        """(atoms to perturb, representative atom of each Hubbard atom, Tr n^{I s} (nhub_atoms, 2)) for
        find_atpert 1 (equal occupations), 2 (species), 3 (space-group orbits) or 4 (all); the classes
        stay in the context for hubbard()'s column reconstruction."""
        nh = self.query_sizes()["nhub_atoms"]
        npert = C.c_int()
        atoms = np.zeros(nh, dtype=np.int32)
        rep = np.zeros(nh, dtype=np.int32)
        tr = np.zeros((nh, 2))
        self._check(lib().hp_perturbed_atoms(self._ptr, int(find_atpert), float(docc_thr), float(dist_thr),
                                             C.byref(npert), _iptr(atoms), _iptr(rep), _dptr(tr)),
                    "hp_perturbed_atoms")
        return [int(a) for a in atoms[:npert.value]], [int(r) for r in rep], tr

    def irreducible_q(self):
        """(q indices to compute under time reversal, partner q of every q)."""
        nq = self.query_sizes()["nq"]
        n = C.c_int()
        iq = np.zeros(nq, dtype=np.int32)
        partner = np.zeros(nq, dtype=np.int32)
        self._check(lib().hp_irreducible_q(self._ptr, C.byref(n), _iptr(iq), _iptr(partner)), "hp_irreducible_q")
        return [int(x) for x in iq[:n.value]], [int(x) for x in partner]

    def irreducible_pairs(self):
        """[(iq, atom)]: the responses to compute under the kept classes and, with find_atpert 3, the
        star of q (hp_irreducible_pairs)."""
        s = self.query_sizes()
        cap = s["nq"] * s["nhub_atoms"]
        n = C.c_int()
        iq = np.zeros(cap, dtype=np.int32)
        at = np.zeros(cap, dtype=np.int32)
        self._check(lib().hp_irreducible_pairs(self._ptr, C.byref(n), _iptr(iq), _iptr(at)), "hp_irreducible_pairs")
        return [(int(a), int(b)) for a, b in zip(iq[:n.value], at[:n.value])]

    def sphere_kq(self, iq, ik):
        """Miller indices (npw, 3) of the k+q sphere in the response's coefficient order."""
        n = C.c_int()
        self._check(lib().hp_sphere_kq(self._ptr, int(iq), int(ik), C.byref(n), None), "hp_sphere_kq")
        m = np.zeros((n.value, 3), dtype=np.int32)
        self._check(lib().hp_sphere_kq(self._ptr, int(iq), int(ik), C.byref(n), _iptr(m)), "hp_sphere_kq")
        return m

    def apply_sternheimer(self, iq, ik, spin, eps, psi):
        """(H_k+q + alpha O_k+q - eps_b) psi_b through the response's own kernels; psi (nb, npw_k+q)."""
        x = np.ascontiguousarray(psi, dtype=np.complex128)
        e = np.ascontiguousarray(eps, dtype=np.float64).reshape(-1)
        out = np.empty_like(x)
        self._check(lib().hp_apply_sternheimer(self._ptr, int(iq), int(ik), int(spin), x.shape[0], _dptr(e),
                                               _dptr(x.view(np.float64)), _dptr(out.view(np.float64))),
                    "hp_apply_sternheimer")
        return out


def batch_band_choice(ctx, w):
    """(b, gap): the band count b in [n_H + n_L, 5 n_H + 3 n_L] of a synthetic batch cell (nspin = 1)
    with the largest gap min_k eps_b(k) - max_k eps_(b-1)(k) of the bare Hamiltonian's spectrum over
    the k mesh (computed by the library), and that gap in Ha (negative: no band count of the range
    is gapped)."""
    kinds = [int(s) for s, _ in w["atoms"]]
    nH = sum(1 for k in kinds if k == 0)
    nL = len(kinds) - nH
    lo, hi = nH + nL, 5 * nH + 3 * nL
    e = np.array([ctx.bare_levels(hi + 1, ik) for ik in range(ctx.query_sizes()["nk"])])
    gap = {n: float(e[:, n].min() - e[:, n - 1].max()) for n in range(lo, hi + 1)}
    b = max(gap, key=gap.get)
    return b, gap[b]


def batch_electron_count(ctx, w):
    """nelec = 2 b for the band count of batch_band_choice."""
    return 2.0 * batch_band_choice(ctx, w)[0]


def batch_run(contexts):
    """Every (q, J) response and chi0, chi, U/V of several independent cells at once, one host
    thread per cell inside the library (each context should carry its own CUDA stream).
    -> list of (chi0, chi, hub) per context."""
    n = len(contexts)
    dims = [c.query_sizes()["nchi"] for c in contexts]
    out = [tuple(np.zeros((m, m)) for _ in range(3)) for m in dims]
    PD = C.POINTER(C.c_double)
    arr = [(PD * n)(*[_dptr(o[j]) for o in out]) for j in range(3)]
    ptrs = (C.c_void_p * n)(*[c._ptr for c in contexts])
    status = np.zeros(n, dtype=np.int32)
    st = lib().hp_batch_run(n, ptrs, arr[0], arr[1], arr[2], _iptr(status))
    if st != HP_OK:
        bad = int(np.nonzero(status)[0][0]) if np.any(status) else 0
        raise HPError(st, "hp_batch_run (cell %d)" % bad, contexts[bad].last_error())
    return out

