"""Thin ctypes binding of libexpgb (include/exp.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; PyTorch supplies
device memory (its caching allocator, through the exp_allocator callbacks) and
the CUDA stream.  There is no CPU fallback: without the built library every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libexpgb.so")

EXP_FP64, EXP_EMU_BF16, EXP_EMU_DS = 0, 1, 2
EXP_GUESS_MP2, EXP_GUESS_USER = 0, 1
STATUS = {0: "EXP_OK", 1: "EXP_EINVAL", 2: "EXP_ENOMEM", 3: "EXP_ECUDA", 4: "EXP_ENOTCONV",
          5: "EXP_ENUMERIC", 6: "EXP_ETIMEOUT", 7: "EXP_ESTATE"}
(EXP_OK, EXP_EINVAL, EXP_ENOMEM, EXP_ECUDA, EXP_ENOTCONV, EXP_ENUMERIC, EXP_ETIMEOUT,
 EXP_ESTATE) = range(8)


class ExpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class Config(C.Structure):
    _fields_ = [("n_inst", C.c_int), ("n_occ", C.c_int), ("n_virt", C.c_int), ("n_irrep", C.c_int),
                ("irrep_occ", C.POINTER(C.c_int32)), ("irrep_virt", C.POINTER(C.c_int32)),
                ("eps_occ", C.POINTER(C.c_double)), ("eps_virt", C.POINTER(C.c_double)),
                ("precision", C.c_int), ("n_slices", C.c_int), ("diis_dim", C.c_int),
                ("conv_tol", C.c_double), ("max_iter", C.c_int), ("guess", C.c_int),
                ("emu_min_macs", C.c_double), ("n_active", C.c_int),
                ("active_virt", C.POINTER(C.c_int32)), ("level_shift", C.c_double),
                ("packed", C.c_int), ("n_slices_major", C.c_int),
                ("denom_shift", C.c_double), ("denom_shift_n", C.c_int), ("real_arith", C.c_int)]


class T3Info(C.Structure):
    _fields_ = [("e_re", C.c_double), ("e_im", C.c_double), ("ms", C.c_double), ("ms_products", C.c_double),
                ("ms_energy", C.c_double), ("macs", C.c_double),
                ("macs_run", C.c_double), ("x_elems", C.c_double), ("n_triples", C.c_int64), ("n_block_triples", C.c_int),
                ("block", C.c_int)]


class IterInfo(C.Structure):
    _fields_ = [("e_re", C.c_double), ("e_im", C.c_double), ("max_dt", C.c_double),
                ("diis_n", C.c_int), ("n_converged", C.c_int), ("ms", C.c_double)]


_lib = None


def lib():
    """Load libexpgb.so (built by paper_2004_03682_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libexpgb.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    L.exp_create.argtypes = [C.POINTER(Config), C.POINTER(Allocator), P, C.POINTER(P)]
    L.exp_destroy.argtypes = [P]
    L.exp_destroy.restype = None
    L.exp_init_integrals.argtypes = [P, C.POINTER(C.c_uint64), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.exp_ccsd_iterate.argtypes = [P, C.c_int, C.POINTER(IterInfo), C.POINTER(C.c_int)]
    L.exp_energy.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.exp_instance_state.argtypes = [P, C.c_int, C.POINTER(C.c_int)]
    L.exp_instance_state.restype = C.c_int
    L.exp_get_amplitudes.argtypes = [P, C.c_int, P, P]
    L.exp_fs_sector_0h1p.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double), C.POINTER(C.c_int)]
    L.exp_fs_sector_0h1p.restype = C.c_int
    L.exp_fs_sector_0h2p.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double), C.POINTER(C.c_int)]
    L.exp_fs_sector_0h2p.restype = C.c_int
    L.exp_set_amplitudes.argtypes = [P, C.c_int, P, P]
    L.exp_work_per_iteration.argtypes = [P, C.POINTER(C.c_double)]
    L.exp_ccsd_t.argtypes = [P, C.c_int, C.c_int, C.POINTER(T3Info), C.POINTER(C.c_double)]
    L.exp_ccsd_t.restype = C.c_int
    L.exp_work_per_iteration.restype = C.c_int
    L.exp_profile_top.argtypes = [P, C.c_int, C.c_char_p, C.c_int, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]
    L.exp_profile_top.restype = C.c_int
    L.exp_zgemm.argtypes = [C.POINTER(Allocator), P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P, P, P,
                            C.c_double, C.c_double, C.c_int]
    L.exp_zgemm.restype = C.c_int
    L.exp_mlp_num_params.argtypes = []
    L.exp_mlp_num_params.restype = C.c_int
    L.exp_mlp_create.argtypes = [C.POINTER(Allocator), P, C.c_uint64, C.c_int, C.POINTER(P)]
    L.exp_mlp_destroy.argtypes = [P]
    L.exp_mlp_destroy.restype = None
    L.exp_mlp_add_training_data.argtypes = [P, P]
    L.exp_mlp_train.argtypes = [P, C.c_int, C.c_int, C.c_double, C.c_uint64, C.POINTER(C.c_double)]
    L.exp_mlp_apply.argtypes = [P, P]
    L.exp_mlp_params.argtypes = [P, C.POINTER(C.c_float), C.POINTER(C.c_float)]
    L.exp_mlp_loss_grad.argtypes = [P, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_float)]
    L.exp_mlp_num_samples.argtypes = [P]
    L.exp_mlp_num_samples.restype = C.c_int64
    L.exp_mlp_eval.argtypes = [P, C.POINTER(C.c_double)]
    L.exp_mlp_samples.argtypes = [P, C.c_int64, C.c_int64, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                  C.POINTER(C.c_float)]
    L.exp_mlp_samples.restype = C.c_int
    L.exp_mlp_eval.restype = C.c_int
    L.exp_mlp_last_error.argtypes = [P]
    L.exp_mlp_last_error.restype = C.c_char_p
    for name in ("exp_mlp_create", "exp_mlp_add_training_data", "exp_mlp_train", "exp_mlp_apply",
                 "exp_mlp_params", "exp_mlp_loss_grad"):
        getattr(L, name).restype = C.c_int
    L.exp_pade_zero.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int, C.c_int,
                                C.POINTER(C.c_double)]
    L.exp_pade_zero.restype = C.c_int
    L.exp_test_emu_wait.argtypes = [C.c_int, C.c_double]
    L.exp_test_emu_wait.restype = C.c_int
    L.exp_kernel_launches.argtypes = [P]
    L.exp_kernel_launches.restype = C.c_int64
    L.exp_last_error.argtypes = [P]
    L.exp_last_error.restype = C.c_char_p
    for name in ("exp_create", "exp_init_integrals", "exp_ccsd_iterate", "exp_energy",
                 "exp_get_amplitudes", "exp_set_amplitudes"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _arr(a, ctype, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.POINTER(ctype))


class TorchAllocator:
    """exp_allocator backed by the PyTorch caching allocator on one stream."""

    def __init__(self, device: int, stream):
        import torch
        self._torch = torch
        self.device = device
        self.stream = stream
        self.live = {}

        def _alloc(nbytes, user):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), device, stream)
            except Exception:
                return None
            self.live[p] = nbytes
            return p

        def _free(ptr, user):
            if ptr in self.live:
                del self.live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self._a = ALLOC_FN(_alloc)
        self._f = FREE_FN(_free)
        self.struct = Allocator(self._a, self._f, None)


class Context:
    """One exp_ctx: n_inst same-sized CCSD instances on one GPU."""

    def __init__(self, n_occ, n_virt, irrep_occ, irrep_virt, eps_occ, eps_virt, n_inst=1,
                 precision=EXP_FP64, n_slices=5, diis_dim=6, conv_tol=1e-9, max_iter=500,
                 guess=EXP_GUESS_MP2, device=0, emu_min_macs=0.0, active=None, level_shift=0.0,
                 packed=True, allocator=None, n_slices_major=0, denom_shift=0.0, denom_shift_n=1,
                 real_arith=False):
        import torch
        self._torch = torch
        L = lib()
        self.L = L
        self.device = device
        self.n_occ, self.n_virt, self.n_inst = int(n_occ), int(n_virt), int(n_inst)
        torch.cuda.set_device(device)
        self.stream = torch.cuda.Stream(device=device)
        # allocator: a factory (device, stream) -> object with a .struct exp_allocator
        self.alloc = (allocator or TorchAllocator)(device, self.stream)
        self._keep = []
        io, pio = _arr(irrep_occ, C.c_int32, np.int32)
        iv, piv = _arr(irrep_virt, C.c_int32, np.int32)
        eo, peo = _arr(np.asarray(eps_occ, dtype=np.float64).reshape(-1), C.c_double, np.float64)
        ev, pev = _arr(np.asarray(eps_virt, dtype=np.float64).reshape(-1), C.c_double, np.float64)
        self._keep += [io, iv, eo, ev]
        self.n_active = 0 if active is None else len(active)
        pa = None
        if self.n_active:
            ac, pa = _arr(np.asarray(active, dtype=np.int32), C.c_int32, np.int32)
            self._keep.append(ac)
        cfg = Config(self.n_inst, self.n_occ, self.n_virt, len(io), pio, piv, peo, pev,
                     int(precision), int(n_slices), int(diis_dim), float(conv_tol), int(max_iter),
                     int(guess), float(emu_min_macs), self.n_active, pa, float(level_shift), int(bool(packed)),
                     int(n_slices_major), float(denom_shift), int(denom_shift_n), int(bool(real_arith)))
        h = C.c_void_p()
        st = L.exp_create(C.byref(cfg), C.byref(self.alloc.struct), C.c_void_p(self.stream.cuda_stream),
                          C.byref(h))
        if st != 0:
            raise ExpError(st, L.exp_last_error(None).decode())
        self.h = h

    def _check(self, st):
        if st != 0:
            raise ExpError(st, self.L.exp_last_error(self.h).decode())

    def init_integrals(self, seeds, scale_mult=None):
        s, ps = _arr(np.asarray(seeds, dtype=np.uint64).reshape(-1), C.c_uint64, np.uint64)
        pm = None
        if scale_mult is not None:
            m, pm = _arr(np.asarray(scale_mult, dtype=np.float64).reshape(-1), C.c_double, np.float64)
        out = np.zeros(self.n_inst)
        self._check(self.L.exp_init_integrals(self.h, ps, pm, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def iterate(self, n_iter, raise_notconv=False, raise_numeric=True):
        info = (IterInfo * max(n_iter, 1))()
        for k in range(n_iter):
            info[k].ms = -1.0
        conv = C.c_int(0)
        st = self.L.exp_ccsd_iterate(self.h, int(n_iter), info, C.byref(conv))
        if (st not in (0, 4, 5)) or (st == 4 and raise_notconv) or (st == 5 and raise_numeric):
            self._check(st)
        recs = []
        for k in range(n_iter):
            r = info[k]
            if r.ms < 0:
                break
            recs.append(dict(e=complex(r.e_re, r.e_im), max_dt=r.max_dt, diis_n=r.diis_n,
                             n_converged=r.n_converged, ms=r.ms))
        return recs, bool(conv.value), st

    def fs_sector_0h1p(self, inst=0):
        """(H_eff, eigenvalues, n_iter, status) of the (0h,1p) sector for instance `inst`."""
        na = self.n_active
        heff = np.zeros(2 * na * na)
        er, ei = np.zeros(na), np.zeros(na)
        nit = C.c_int(0)
        dp = C.POINTER(C.c_double)
        st = self.L.exp_fs_sector_0h1p(self.h, int(inst), heff.ctypes.data_as(dp), er.ctypes.data_as(dp),
                                       ei.ctypes.data_as(dp), C.byref(nit))
        if st not in (0, 4):
            self._check(st)
        H = (heff[0::2] + 1j * heff[1::2]).reshape(na, na)
        return H, er + 1j * ei, nit.value, st

    def ccsd_t(self, inst=0, per_triple=False, block=0):
        """(T) correction of instance `inst` from its current amplitudes: (E(T), info dict,
        per-triple energies or None).  The per-triple array holds the energy of each i<j<k
        at index C(k,3) + C(j,2) + i.  block: occupied spinors per block (0: automatic)."""
        info = T3Info()
        n3 = self.n_occ * (self.n_occ - 1) * (self.n_occ - 2) // 6
        buf = np.zeros(2 * max(n3, 1)) if per_triple else None
        ptr = buf.ctypes.data_as(C.POINTER(C.c_double)) if per_triple else None
        self._check(self.L.exp_ccsd_t(self.h, int(inst), int(block), C.byref(info), ptr))
        d = {k: getattr(info, k) for k, _ in T3Info._fields_}
        e3 = (buf[0:2 * n3:2] + 1j * buf[1:2 * n3:2]) if per_triple else None
        return complex(info.e_re, info.e_im), d, e3

    def fs_sector_0h2p(self, inst=0):
        """(H_eff over the active pairs x<y, eigenvalues, n_iter, status) of the (0h,2p) sector."""
        na = self.n_active
        npr = na * (na - 1) // 2
        heff = np.zeros(2 * max(npr * npr, 1))
        er, ei = np.zeros(max(npr, 1)), np.zeros(max(npr, 1))
        nit = C.c_int(0)
        dp = C.POINTER(C.c_double)
        st = self.L.exp_fs_sector_0h2p(self.h, int(inst), heff.ctypes.data_as(dp), er.ctypes.data_as(dp),
                                       ei.ctypes.data_as(dp), C.byref(nit))
        if st not in (0, 4):
            self._check(st)
        H = (heff[0:2 * npr * npr:2] + 1j * heff[1:2 * npr * npr:2]).reshape(npr, npr)
        return H, er[:npr] + 1j * ei[:npr], nit.value, st

    def state(self, inst=0) -> int:
        """0 iterating, 1 converged, 2 failed."""
        v = C.c_int()
        self._check(self.L.exp_instance_state(self.h, int(inst), C.byref(v)))
        return v.value

    def energy(self, inst=0) -> complex:
        re, im = C.c_double(), C.c_double()
        self._check(self.L.exp_energy(self.h, int(inst), C.byref(re), C.byref(im)))
        return complex(re.value, im.value)

    def get_amplitudes(self, inst=0):
        torch = self._torch
        o, v = self.n_occ, self.n_virt
        with torch.cuda.stream(self.stream):
            t1 = torch.empty((o, v), dtype=torch.complex128, device=f"cuda:{self.device}")
            t2 = torch.empty((o, o, v, v), dtype=torch.complex128, device=f"cuda:{self.device}")
        self._check(self.L.exp_get_amplitudes(self.h, int(inst), C.c_void_p(t1.data_ptr()),
                                              C.c_void_p(t2.data_ptr())))
        return t1, t2

    def set_amplitudes(self, inst, t1, t2):
        torch = self._torch
        t1 = t1.to(device=f"cuda:{self.device}", dtype=torch.complex128).contiguous()
        t2 = t2.to(device=f"cuda:{self.device}", dtype=torch.complex128).contiguous()
        self.stream.wait_stream(torch.cuda.current_stream())
        self._check(self.L.exp_set_amplitudes(self.h, int(inst), C.c_void_p(t1.data_ptr()),
                                              C.c_void_p(t2.data_ptr())))

    def work_per_iteration(self) -> float:
        """Complex multiply-adds of one iteration (all contractions, all instances)."""
        m = C.c_double()
        self._check(self.L.exp_work_per_iteration(self.h, C.byref(m)))
        return m.value

    def profile_top(self, reps=5, site=None):
        """(site, ms per launch, complex MACs per launch) of the largest contraction, or
        of the contraction at call site `site`."""
        buf = C.create_string_buffer((site or "").encode(), 64)
        ms, macs = C.c_double(), C.c_double()
        self._check(self.L.exp_profile_top(self.h, int(reps), buf, 64, C.byref(ms), C.byref(macs)))
        return buf.value.decode(), ms.value, macs.value

    @property
    def launches(self) -> int:
        return int(self.L.exp_kernel_launches(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.L.exp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """The learned T2 guess (exp_mlp_*)."""

    def __init__(self, seed=0, bf16=True, device=0, stream=None):
        import torch
        self._torch = torch
        self.L = lib()
        torch.cuda.set_device(device)
        self.stream = stream or torch.cuda.Stream(device=device)
        self.alloc = TorchAllocator(device, self.stream)
        h = C.c_void_p()
        st = self.L.exp_mlp_create(C.byref(self.alloc.struct), C.c_void_p(self.stream.cuda_stream), int(seed),
                                   int(bool(bf16)), C.byref(h))
        if st != 0:
            raise ExpError(st, self.L.exp_mlp_last_error(None).decode())
        self.h = h
        self.n_params = self.L.exp_mlp_num_params()

    def _check(self, st):
        if st != 0:
            raise ExpError(st, self.L.exp_mlp_last_error(self.h).decode())

    def add_training_data(self, ctx):
        self._check(self.L.exp_mlp_add_training_data(self.h, ctx.h))

    def train(self, epochs, batch=65536, lr=1e-3, seed=0):
        out = np.zeros(max(epochs, 1))
        self._check(self.L.exp_mlp_train(self.h, int(epochs), int(batch), float(lr), int(seed),
                                         out.ctypes.data_as(C.POINTER(C.c_double))))
        return out[:epochs]

    def apply(self, ctx):
        self._check(self.L.exp_mlp_apply(self.h, ctx.h))

    @property
    def n_samples(self):
        return int(self.L.exp_mlp_num_samples(self.h))

    def samples(self, first=0, count=None):
        n = self.n_samples - first if count is None else count
        x = np.zeros((n, 3), np.float32)
        tm = np.zeros((n, 2), np.float32)
        tg = np.zeros((n, 2), np.float32)
        fp = C.POINTER(C.c_float)
        self._check(self.L.exp_mlp_samples(self.h, int(first), int(n), x.ctypes.data_as(fp), tm.ctypes.data_as(fp),
                                           tg.ctypes.data_as(fp)))
        return x, tm[:, 0] + 1j * tm[:, 1], tg[:, 0] + 1j * tg[:, 1]

    def eval(self):
        v = C.c_double()
        self._check(self.L.exp_mlp_eval(self.h, C.byref(v)))
        return v.value

    def params(self, set=None):
        get = np.zeros(self.n_params, np.float32)
        ps = None
        if set is not None:
            s_ = np.ascontiguousarray(set, dtype=np.float32)
            ps = s_.ctypes.data_as(C.POINTER(C.c_float))
        self._check(self.L.exp_mlp_params(self.h, get.ctypes.data_as(C.POINTER(C.c_float)), ps))
        return get

    def loss_grad(self, x, tmp2, target):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(np.stack([tmp2.real, tmp2.imag], -1), dtype=np.float64)
        g_ = np.ascontiguousarray(np.stack([target.real, target.imag], -1), dtype=np.float64)
        loss = C.c_double()
        grad = np.zeros(self.n_params, np.float32)
        self._check(self.L.exp_mlp_loss_grad(self.h, len(x), x.ctypes.data_as(C.POINTER(C.c_float)),
                                             t.ctypes.data_as(C.POINTER(C.c_double)),
                                             g_.ctypes.data_as(C.POINTER(C.c_double)), C.byref(loss),
                                             grad.ctypes.data_as(C.POINTER(C.c_float))))
        return loss.value, grad

    def close(self):
        if getattr(self, "h", None):
            self.L.exp_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def zgemm(A, B, C=None, alpha=1.0, beta=False, precision=EXP_FP64, n_slices=5):
    """C = alpha A B (+ C) for complex128 CUDA tensors through exp_zgemm."""
    import torch
    L = lib()
    M, K = A.shape
    K2, N = B.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    A = A.contiguous()
    B = B.contiguous()
    Cm = torch.zeros((M, N), dtype=torch.complex128, device=A.device) if C is None else C
    dev = A.device.index or 0
    stream = torch.cuda.current_stream(dev)
    alloc = TorchAllocator(dev, stream)
    a = complex(alpha)
    st = L.exp_zgemm(_byref(alloc.struct), _vp(stream.cuda_stream), int(precision), int(n_slices),
                     int(M), int(N), int(K), _vp(A.data_ptr()), _vp(B.data_ptr()), _vp(Cm.data_ptr()),
                     a.real, a.imag, int(bool(beta)))
    if st != 0:
        raise ExpError(st, L.exp_last_error(None).decode())
    return Cm


def pade_zero(x, values, L, M) -> complex:
    """E(0) of the [L/M] Pade fit of complex values at scales x (exp_pade_zero, host)."""
    Lb = lib()
    xa = np.ascontiguousarray(x, dtype=np.float64)
    v = np.asarray(values, dtype=np.complex128)
    va = np.ascontiguousarray(np.stack([v.real, v.imag], -1).reshape(-1))
    out = np.zeros(2)
    dp = C.POINTER(C.c_double)
    st = Lb.exp_pade_zero(len(xa), xa.ctypes.data_as(dp), va.ctypes.data_as(dp), int(L), int(M),
                          out.ctypes.data_as(dp))
    if st != 0:
        raise ExpError(st, Lb.exp_last_error(None).decode())
    return complex(out[0], out[1])


def _byref(x):
    return C.byref(x)


def _vp(x):
    return C.c_void_p(x)


def from_problems(probs, **kw) -> Context:
    """Context for one or more synthetic problems of the same sizes and irrep split."""
    p0 = probs[0]
    eo = np.stack([p.eps_occ for p in probs])
    ev = np.stack([p.eps_virt for p in probs])
    return Context(p0.n_occ, p0.n_virt, p0.irrep_occ, p0.irrep_virt, eo, ev, n_inst=len(probs), **kw)
