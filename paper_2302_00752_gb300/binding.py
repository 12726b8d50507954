"""Python binding of the C ABI in include/sparse_spectral.h (ctypes).

Argument marshalling only: tensors are passed as device pointers on the
current torch CUDA stream, every computation runs in the library's kernels.
The library must have been built (``paper_2302_00752_gb300.build``); importing
this module without it raises, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsparse_spectral.so")

SS_FP64, SS_FP32, SS_DF64 = 0, 1, 2
STATUS = {0: "SS_OK", 1: "SS_ERR_INVALID", 2: "SS_ERR_OOM", 3: "SS_ERR_CUDA", 4: "SS_ERR_NOT_RECONSTRUCTING",
          5: "SS_ERR_HASH_FULL", 6: "SS_ERR_NOT_ELLIPTIC", 7: "SS_ERR_NOT_CONVERGED", 8: "SS_ERR_TIMEOUT",
          9: "SS_ERR_KEY_RANGE"}


class SSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class Lattice(C.Structure):
    _fields_ = [("d", C.c_int32), ("M", C.c_int64), ("z", C.POINTER(C.c_int64))]


class Trig(C.Structure):
    _fields_ = [("d", C.c_int32), ("n_terms", C.c_int64), ("freq", C.c_void_p), ("coef", C.c_void_p)]


class Sparse(C.Structure):
    _fields_ = [("d", C.c_int32), ("n", C.c_int64), ("freq", C.c_void_p), ("val", C.c_void_p)]


class LatticeSpec(C.Structure):
    _fields_ = [("kind", C.c_int32), ("d", C.c_int32), ("z", C.POINTER(C.c_int64)), ("M", C.c_int64),
                ("raw", C.POINTER(C.c_int64)), ("n_raw", C.c_int32), ("M_min", C.c_int64), ("sigma", C.c_double)]


class SolveStats(C.Structure):
    _fields_ = [("status", C.c_int32), ("outer_iters", C.c_int32), ("inner_iters", C.c_int32),
                ("applies", C.c_int32), ("rel_residual", C.c_double), ("kernel_ms", C.c_double),
                ("half_system", C.c_int32), ("real_coefficients", C.c_int32)]

    def as_dict(self):
        return {"status": STATUS.get(self.status, self.status), "outer_iters": self.outer_iters,
                "inner_iters": self.inner_iters, "applies": self.applies, "rel_residual": self.rel_residual,
                "kernel_ms": self.kernel_ms, "half_system": bool(self.half_system),
                "real_coefficients": bool(self.real_coefficients)}


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run python -m paper_2302_00752_gb300.build)")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    P = C.POINTER
    sigs = {
        "ss_last_error": (C.c_char_p, []),
        "ss_version": (C.c_char_p, []),
        "ss_alloc_count": (C.c_int64, []),
        "ss_profile": (i32, [i32]),
        "ss_profile_entry": (i32, [i32, C.c_char_p, i32, P(i64), P(dbl), P(i32)]),
        "ss_profile_trace": (i32, [i32, C.c_char_p, i32, P(dbl), P(dbl), P(i32)]),
        "solve_set_wait_limit": (i32, [vp, i64]),
        "stamp_set_table_limit": (i32, [i64]),
        "lattice_size": (i32, [i64, i64, dbl, i64, P(i64)]),
        "lattice_check": (i32, [P(Lattice), vp, i64, vp]),
        "lattice_random": (i32, [vp, i64, i32, dbl, i64, P(i64), i32, P(i64), P(i64), P(i32), vp]),
        "lattice_random_smooth": (i32, [vp, i64, i32, dbl, i64, P(i64), i32, P(i64), P(i64), P(i32), vp]),
        "lattice_cbc": (i32, [vp, i64, i32, i64, P(i64), i32, P(i64), P(i64), vp]),
        "lattice_sample": (i32, [P(Lattice), P(Trig), i32, vp, vp]),
        "sft_recover_samples": (i32, [P(Lattice), vp, i32, vp, i64, i64, dbl, vp, vp, P(i64), vp]),
        "sft_recover": (i32, [P(Lattice), P(Trig), i32, vp, i64, i64, dbl, vp, vp, P(i64), vp]),
        "sft_identify": (i32, [P(Lattice), P(Trig), i32, i32, i64, dbl, vp, vp, P(i64), vp]),
        "sft_identify_samples": (i32, [P(Lattice), i32, vp, i32, i64, dbl, i64, i32, vp, vp, P(i64), vp]),
        "stamp_build": (i32, [P(Sparse), vp, i64, i32, P(vp), vp]),
        "stamp_build_adr": (i32, [P(Sparse), P(Sparse), P(Sparse), vp, i64, i32, P(vp), vp]),
        "stamp_info": (i32, [vp, P(i64), P(i64), P(i64), P(i32)]),
        "stamp_real_coefficients": (i32, [vp, P(i32)]),
        "stamp_export": (i32, [vp, vp, vp, vp]),
        "stamp_lookup": (i32, [vp, vp, i64, vp, vp]),
        "stamp_scatter": (i32, [vp, P(Sparse), vp, P(i64), vp]),
        "stamp_destroy": (None, [vp]),
        "stamp_extend": (i32, [vp, i32, vp]),
        "proxy_residual": (i32, [vp, vp, i64, vp, P(dbl), vp]),
        "proxy_mc": (i32, [vp, vp, i64, P(Trig), vp, i64, vp, vp, vp]),
        "galerkin_apply": (i32, [vp, vp, vp, i32, vp]),
        "solve": (i32, [vp, vp, vp, dbl, i32, i32, P(SolveStats), vp]),
        "solve_set_config": (i32, [vp, i32, i32, i32]),
        "solve_set_symmetry": (i32, [vp, i32]),
        "solve_noalloc": (i32, [vp, vp, vp, dbl, i32, i32, P(SolveStats), vp]),
        "batch_create": (i32, [i32, P(vp), P(vp), vp]),
        "batch_solve": (i32, [vp, P(vp), P(vp), dbl, i32, i32, i32, P(SolveStats), vp]),
        "batch_autotune": (i32, [vp, P(vp), P(vp), dbl, i32, i32, P(dbl), vp]),
        "batch_config": (i32, [vp, P(i32), P(i32), P(i32), P(i32), P(i32)]),
        "batch_set_config": (i32, [vp, i32, i32, i32]),
        "batch_set_symmetry": (i32, [vp, i32]),
        "batch_destroy": (None, [vp]),
        "sparse_spectral_solve": (i32, [P(LatticeSpec), P(Trig), P(Trig), vp, i64, i32, dbl, i32, i32, dbl, i32,
                                        P(i64), P(i64), P(vp), vp, i64, P(SolveStats), vp]),
        "stamp_solution": (i32, [vp, vp, vp]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _check(status):
    if status != 0:
        raise SSError(status, lib.ss_last_error().decode(errors="replace"))


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


def _dev_i32(x, d=None):
    # device tensors that already have the layout are passed through untouched
    # (each torch call costs host time on the path between two library calls)
    if (torch.is_tensor(x) and x.is_cuda and x.dtype == torch.int32 and x.is_contiguous()
            and x.device.index == torch.cuda.current_device()):
        t = x
    else:
        t = torch.as_tensor(np.asarray(x) if not torch.is_tensor(x) else x)
        t = t.to(device="cuda", dtype=torch.int32).contiguous()
    if d is not None and (t.dim() != 2 or t.shape[1] != d):
        t = t.reshape(-1, d)
    return t


def _dev_c128(x):
    if (torch.is_tensor(x) and x.is_cuda and x.dtype == torch.complex128 and x.is_contiguous()
            and x.device.index == torch.cuda.current_device()):
        return x
    t = x if torch.is_tensor(x) else torch.as_tensor(np.asarray(x, dtype=np.complex128))
    return t.to(device="cuda", dtype=torch.complex128).contiguous()


def _lattice(z, M):
    z = np.ascontiguousarray(np.asarray(z, dtype=np.int64))
    arr = (C.c_int64 * len(z))(*z.tolist())
    lat = Lattice(len(z), int(M), arr)
    lat._keep = arr
    return lat


def _prec(p):
    if p in (SS_FP64, "fp64", "float64"):
        return SS_FP64
    if p in (SS_FP32, "fp32", "float32", "fp32_refined"):
        return SS_FP32
    if p in (SS_DF64, "df64"):
        return SS_DF64
    raise ValueError(f"unknown precision {p!r}")


def version():
    return lib.ss_version().decode()


# ------------------------------------------------------------------ lattice

def lattice_size(K, n_I, sigma=0.05, M_min=0):
    M = C.c_int64()
    _check(lib.lattice_size(int(K), int(n_I), float(sigma), int(M_min), C.byref(M)))
    return M.value


def lattice_check(z, M, freq):
    f = _dev_i32(freq, len(z))
    lat = _lattice(z, M)
    _check(lib.lattice_check(C.byref(lat), _ptr(f), f.shape[0], _stream()))


def lattice_random(freq, raw, sigma=0.05, M_min=0, smooth=False):
    """Random rank-1 lattice (Lemma RandomRank1Lattice): prime M, or with
    smooth=True the FFT-friendly 7-smooth M (lattice_random_smooth)."""
    raw = np.ascontiguousarray(np.asarray(raw, dtype=np.int64))
    attempts, d = raw.shape
    f = _dev_i32(freq, d)
    z = (C.c_int64 * d)()
    M = C.c_int64()
    att = C.c_int32()
    fn = lib.lattice_random_smooth if smooth else lib.lattice_random
    _check(fn(_ptr(f), f.shape[0], d, float(sigma), int(M_min), raw.ctypes.data_as(C.POINTER(C.c_int64)), attempts,
              z, C.byref(M), C.byref(att), _stream()))
    return np.array(z[:], dtype=np.int64), M.value, att.value


def lattice_cbc(freq, raw, M_min):
    raw = np.ascontiguousarray(np.asarray(raw, dtype=np.int64))
    d, n_cand = raw.shape
    f = _dev_i32(freq, d)
    z = (C.c_int64 * d)()
    M = C.c_int64()
    _check(lib.lattice_cbc(_ptr(f), f.shape[0], d, int(M_min), raw.ctypes.data_as(C.POINTER(C.c_int64)), n_cand,
                           z, C.byref(M), _stream()))
    return np.array(z[:], dtype=np.int64), M.value


# ---------------------------------------------------------------------- SFT

def _trig(freq, coef, d):
    f = _dev_i32(freq, d)
    c = _dev_c128(coef)
    t = Trig(d, f.shape[0], _ptr(f), _ptr(c))
    t._keep = (f, c)
    return t


def lattice_sample(z, M, freq, coef, precision="fp64"):
    p = _prec(precision)
    lat = _lattice(z, M)
    g = _trig(freq, coef, len(z))
    out = torch.empty(int(M), dtype=torch.float64 if p == SS_FP64 else torch.float32, device="cuda")
    _check(lib.lattice_sample(C.byref(lat), C.byref(g), p, _ptr(out), _stream()))
    return out


def _recover_out(cand, d):
    fo = torch.empty((cand.shape[0], d), dtype=torch.int32, device="cuda")
    vo = torch.empty(cand.shape[0], dtype=torch.complex128, device="cuda")
    return fo, vo


def sft_recover_samples(z, M, samples, cand, s_max=0, tau=1e-9, precision="fp64"):
    p = _prec(precision)
    lat = _lattice(z, M)
    cd = _dev_i32(cand, len(z))
    fo, vo = _recover_out(cd, len(z))
    n = C.c_int64()
    _check(lib.sft_recover_samples(C.byref(lat), _ptr(samples), p, _ptr(cd), cd.shape[0], int(s_max), float(tau),
                                   _ptr(fo), _ptr(vo), C.byref(n), _stream()))
    return fo[: n.value], vo[: n.value]


def sft_recover(z, M, freq, coef, cand, s_max=0, tau=1e-9, precision="fp64"):
    p = _prec(precision)
    lat = _lattice(z, M)
    g = _trig(freq, coef, len(z))
    cd = _dev_i32(cand, len(z))
    fo, vo = _recover_out(cd, len(z))
    n = C.c_int64()
    _check(lib.sft_recover(C.byref(lat), C.byref(g), p, _ptr(cd), cd.shape[0], int(s_max), float(tau), _ptr(fo),
                           _ptr(vo), C.byref(n), _stream()))
    return fo[: n.value], vo[: n.value]


def sft_identify(z, M, freq, coef, P, s_max, tau=1e-9, precision="fp64"):
    """Support identification from the d shifted lattices x_j + e_i / P
    (P > 2 max |k_i|); returns (freq, val) with each k followed by -k."""
    p = _prec(precision)
    lat = _lattice(z, M)
    d = len(z)
    g = _trig(freq, coef, d)
    fo = torch.empty((int(s_max), d), dtype=torch.int32, device="cuda")
    vo = torch.empty(int(s_max), dtype=torch.complex128, device="cuda")
    n = C.c_int64()
    _check(lib.sft_identify(C.byref(lat), C.byref(g), p, int(P), int(s_max), float(tau), _ptr(fo), _ptr(vo),
                            C.byref(n), _stream()))
    return fo[: n.value], vo[: n.value]


def sft_identify_samples(z, M, samples, P, s_max, tau=1e-9, keep=0, robust=False, precision="fp64"):
    """Identification from given samples ((d+1) x M: the lattice, then the d
    shifted lattices); keep / robust for compressible data."""
    p = _prec(precision)
    lat = _lattice(z, M)
    d = len(z)
    dt = torch.float64 if p == SS_FP64 else torch.float32
    x = samples if torch.is_tensor(samples) else torch.as_tensor(np.asarray(samples))
    x = x.to(device="cuda", dtype=dt).contiguous()
    if x.shape != (d + 1, int(M)):
        raise ValueError("samples must be (d + 1) x M")
    fo = torch.empty((int(s_max), d), dtype=torch.int32, device="cuda")
    vo = torch.empty(int(s_max), dtype=torch.complex128, device="cuda")
    n = C.c_int64()
    _check(lib.sft_identify_samples(C.byref(lat), int(P), _ptr(x), p, int(s_max), float(tau), int(keep),
                                    int(bool(robust)), _ptr(fo), _ptr(vo), C.byref(n), _stream()))
    return fo[: n.value], vo[: n.value]


# -------------------------------------------------------------------- stamp

class Stamp:
    """S^N[a_hat](F) on the device (owns the library handle)."""

    def __init__(self, handle, d):
        self._h = C.c_void_p(handle)
        self.d = d
        size, nnz, zero = C.c_int64(), C.c_int64(), C.c_int64()
        lv = C.c_int32()
        _check(lib.stamp_info(self._h, C.byref(size), C.byref(nnz), C.byref(zero), C.byref(lv)))
        self.size, self.nnz, self.zero_index, self.n_levels = size.value, nnz.value, zero.value, lv.value

    @property
    def real_coefficients(self):
        """a_hat taken as real (real entry coefficients, see stamp_real_coefficients)."""
        r = C.c_int32()
        _check(lib.stamp_real_coefficients(self.handle, C.byref(r)))
        return bool(r.value)

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("stamp destroyed")
        return self._h

    def export(self):
        freq = torch.empty((self.size, self.d), dtype=torch.int32, device="cuda")
        level = torch.empty(self.size, dtype=torch.int8, device="cuda")
        _check(lib.stamp_export(self.handle, _ptr(freq), _ptr(level), _stream()))
        return freq, level

    def lookup(self, freq):
        f = _dev_i32(freq, self.d)
        idx = torch.empty(f.shape[0], dtype=torch.int64, device="cuda")
        _check(lib.stamp_lookup(self.handle, _ptr(f), f.shape[0], _ptr(idx), _stream()))
        return idx

    def scatter(self, freq, val, count_outside=True):
        """(values on S, number of input frequencies outside S); without the
        count the call stays asynchronous (count returned as None)."""
        f = _dev_i32(freq, self.d)
        v = _dev_c128(val)
        sp = Sparse(self.d, f.shape[0], _ptr(f), _ptr(v))
        out = torch.empty(self.size, dtype=torch.complex128, device="cuda")
        outside = C.c_int64()
        _check(lib.stamp_scatter(self.handle, C.byref(sp), _ptr(out), C.byref(outside) if count_outside else None,
                                 _stream()))
        return out, (outside.value if count_outside else None)

    def extend(self, levels=1):
        """Grow S^N to S^{N+levels} in place (existing indices unchanged)."""
        _check(lib.stamp_extend(self.handle, int(levels), _stream()))
        size, nnz, zero = C.c_int64(), C.c_int64(), C.c_int64()
        lv = C.c_int32()
        _check(lib.stamp_info(self._h, C.byref(size), C.byref(nnz), C.byref(zero), C.byref(lv)))
        self.size, self.nnz, self.zero_index, self.n_levels = size.value, nnz.value, zero.value, lv.value
        return self

    def set_wait_limit(self, ns):
        """Bound (ns) on each device-side wait of this stamp's solver (0: give up at once)."""
        _check(lib.solve_set_wait_limit(self.handle, int(ns)))

    def set_symmetry(self, use_half):
        """Solve real data through the Hermitian half system (default True)."""
        _check(lib.solve_set_symmetry(self.handle, int(bool(use_half))))

    def set_solve_config(self, block, blocks_per_sm, chunks_per_block):
        """Tile shape of the persistent solve (see solve_set_config)."""
        _check(lib.solve_set_config(self.handle, int(block), int(blocks_per_sm), int(chunks_per_block)))

    def destroy(self):
        if self._h:
            lib.stamp_destroy(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.destroy()


def stamp_build(a_freq, a_val, f_freq, N):
    af = torch.as_tensor(a_freq) if torch.is_tensor(a_freq) else torch.as_tensor(np.asarray(a_freq))
    d = int(af.shape[1])
    af = _dev_i32(af, d)
    av = _dev_c128(a_val)
    ff = _dev_i32(f_freq, d)
    sp = Sparse(d, af.shape[0], _ptr(af), _ptr(av))
    h = C.c_void_p()
    _check(lib.stamp_build(C.byref(sp), _ptr(ff), ff.shape[0], int(N), C.byref(h), _stream()))
    return Stamp(h.value, d)


def _sparse(freq, val, d):
    f = _dev_i32(np.asarray(freq).reshape(-1, d) if not torch.is_tensor(freq) else freq, d)
    v = _dev_c128(val)
    sp = Sparse(d, f.shape[0], _ptr(f) if f.numel() else None, _ptr(v) if v.numel() else None)
    sp._keep = (f, v)
    return sp


def stamp_build_adr(a_freq, a_val, b, c_freq, c_val, f_freq, N):
    """Stamping set and operator of -div(a grad u) + b.grad u + c u = f
    (Remark ADR); b: d pairs (freq, val), one per component of b."""
    af = np.asarray(a_freq.cpu() if torch.is_tensor(a_freq) else a_freq)
    d = int(af.shape[1])
    if len(b) != d:
        raise ValueError("b needs one (freq, val) pair per coordinate")
    sa = _sparse(a_freq, a_val, d)
    sc = _sparse(c_freq, c_val, d)
    sb = (Sparse * d)()
    keep = []
    for j, (bf, bv) in enumerate(b):
        one = _sparse(bf, bv, d)
        sb[j] = one
        keep.append(one._keep)
    ff = _dev_i32(f_freq, d)
    h = C.c_void_p()
    _check(lib.stamp_build_adr(C.byref(sa), sb, C.byref(sc), _ptr(ff), ff.shape[0], int(N), C.byref(h), _stream()))
    st = Stamp(h.value, d)
    st.adr = True
    return st


def proxy_residual(stamp, u_prefix, f_on_S):
    """(||f - L u||^2, ||f||^2) over S with u on the first len(u_prefix) frequencies."""
    u = _dev_c128(u_prefix)
    f = _dev_c128(f_on_S)
    out = (C.c_double * 2)()
    _check(lib.proxy_residual(stamp.handle, _ptr(u), u.numel(), _ptr(f), out, _stream()))
    return out[0], out[1]


def proxy_mc(stamp, u_prefix, f_freq, f_coef, X):
    """Point values (r, f) of the Monte Carlo proxy at x = X / 2^32 (X uint32
    [Q, d], numpy or tensor); the estimate is sqrt(sum r^2 / sum f^2)."""
    u = _dev_c128(u_prefix)
    g = _trig(f_freq, f_coef, stamp.d)
    Xn = X.cpu().numpy() if torch.is_tensor(X) else np.asarray(X)
    Xd = torch.from_numpy(np.ascontiguousarray(Xn.astype(np.uint32)).view(np.int32)).cuda()
    Q = int(Xd.shape[0]) if Xd.dim() == 2 else 0
    r = torch.empty(Q, dtype=torch.float64, device="cuda")
    f = torch.empty(Q, dtype=torch.float64, device="cuda")
    _check(lib.proxy_mc(stamp.handle, _ptr(u), u.numel(), C.byref(g), _ptr(Xd), Q, _ptr(r), _ptr(f), _stream()))
    return r, f


def galerkin_apply(stamp, u, precision=None):
    if precision is None:
        precision = "fp32" if u.dtype == torch.complex64 else "fp64"
    p = _prec(precision)
    dt = torch.complex128 if p == SS_FP64 else torch.complex64
    u = u.to(device="cuda", dtype=dt).contiguous()
    y = torch.empty_like(u)
    _check(lib.galerkin_apply(stamp.handle, _ptr(u), _ptr(y), p, _stream()))
    return y


def _check_solution_buffer(t, n, name):
    if not (torch.is_tensor(t) and t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous complex128 CUDA tensor")
    if t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements; the stamping set has {n}")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{torch.cuda.current_device()}")


def set_table_limit(max_slots):
    """Slot bound of the hash tables of stamps built from now on (0: none)."""
    _check(lib.stamp_set_table_limit(int(max_slots)))


def profile(on, level=2):
    """Start (True) or stop kernel timing; resets the totals.  level 1: the
    main kernels only (little host work per step), 2: every bracket."""
    _check(lib.ss_profile(int(level) if on else 0))


def profile_totals():
    """{kernel name: (launches, total ms)} accumulated since profile(True)."""
    n = C.c_int32(0)
    out = {}
    i = 0
    while True:
        name = C.create_string_buffer(128)
        cnt, ms = C.c_int64(), C.c_double()
        if lib.ss_profile_entry(i, name, 128, C.byref(cnt), C.byref(ms), C.byref(n)) != 0:
            break
        out[name.value.decode()] = (cnt.value, ms.value)
        i += 1
    return out



def profile_trace():
    """[(name, start ms, end ms)] of the brackets since profile(True), device
    time relative to the first bracket's start."""
    out = []
    n = C.c_int32(0)
    lib.ss_profile_trace(0, None, 0, None, None, C.byref(n))
    name = C.create_string_buffer(128)
    a, b = C.c_double(), C.c_double()
    for i in range(n.value):
        _check(lib.ss_profile_trace(i, name, 128, C.byref(a), C.byref(b), None))
        out.append((name.value.decode(), a.value, b.value))
    return out

def alloc_count():
    """Allocation calls the library has made in this process (diagnostic)."""
    return int(lib.ss_alloc_count())


def solve(stamp, f_on_S, tol=1e-12, max_iter=1000, precision="fp64", out=None, raise_on_error=True):
    f = _dev_c128(f_on_S)
    if f.numel() != stamp.size:
        raise ValueError(f"f_on_S has {f.numel()} elements; the stamping set has {stamp.size}")
    if out is None:
        u = torch.empty_like(f)
    else:
        _check_solution_buffer(out, stamp.size, "out")
        u = out
    st = SolveStats()
    status = lib.solve(stamp.handle, _ptr(f), _ptr(u), float(tol), int(max_iter), _prec(precision), C.byref(st),
                       _stream())
    if raise_on_error:
        _check(status)
    return u, st.as_dict()


def solve_noalloc(stamp, f_on_S, out, tol=1e-12, max_iter=1000, precision="fp64"):
    """Allocation-free solve: for callers that must not allocate device memory
    while they run (plug-ins in a host application that owns all device
    memory, loops that must not stall on an allocation, fixed memory
    budgets).  ``f_on_S`` and ``out`` are caller-owned complex128
    device tensors of length |S|; the workspace is a fixed library array for
    |S| <= 32768 (larger sets raise SSError).  Calls that overlap on the GPU
    share that array and race."""
    _check_solution_buffer(f_on_S, stamp.size, "f_on_S")
    _check_solution_buffer(out, stamp.size, "out")
    st = SolveStats()
    _check(lib.solve_noalloc(stamp.handle, _ptr(f_on_S), _ptr(out), float(tol), int(max_iter), _prec(precision),
                             C.byref(st), _stream()))
    return out, st.as_dict()


# -------------------------------------------------------------------- batch

class Batch:
    """Many stamps solved by one persistent launch."""

    def __init__(self, stamps):
        self.stamps = list(stamps)
        arr = (C.c_void_p * len(self.stamps))(*[s.handle.value for s in self.stamps])
        h = C.c_void_p()
        _check(lib.batch_create(len(self.stamps), arr, C.byref(h), _stream()))
        self._h = h

    def _ptr_arrays(self, fs, us):
        fa = (C.c_void_p * len(fs))(*[f.data_ptr() for f in fs])
        ua = (C.c_void_p * len(us))(*[u.data_ptr() for u in us])
        return fa, ua

    def solve(self, fs, us=None, tol=1e-12, max_iter=1000, precision="fp32", use_graph=True):
        fs = [_dev_c128(f) for f in fs]
        us = [torch.empty_like(f) for f in fs] if us is None else us
        fa, ua = self._ptr_arrays(fs, us)
        st = (SolveStats * len(fs))()
        _check(lib.batch_solve(self._h, fa, ua, float(tol), int(max_iter), _prec(precision), int(bool(use_graph)),
                               st, _stream()))
        return us, [s.as_dict() for s in st]

    def autotune(self, fs, us=None, tol=1e-12, max_iter=1000, precision="fp32"):
        fs = [_dev_c128(f) for f in fs]
        us = [torch.empty_like(f) for f in fs] if us is None else us
        fa, ua = self._ptr_arrays(fs, us)
        best = C.c_double()
        _check(lib.batch_autotune(self._h, fa, ua, float(tol), int(max_iter), _prec(precision), C.byref(best),
                                  _stream()))
        return best.value, self.config()

    def config(self):
        v = [C.c_int32() for _ in range(5)]
        _check(lib.batch_config(self._h, *[C.byref(x) for x in v]))
        return dict(zip(["block", "blocks_per_sm", "chunks_per_block", "grid", "n_chunks"], [x.value for x in v]))

    def set_config(self, block, blocks_per_sm, chunks_per_block):
        _check(lib.batch_set_config(self._h, int(block), int(blocks_per_sm), int(chunks_per_block)))

    def set_symmetry(self, use_half):
        """Solve real data through the instances' Hermitian half systems (default True)."""
        _check(lib.batch_set_symmetry(self._h, int(bool(use_half))))

    def destroy(self):
        if self._h:
            lib.batch_destroy(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ------------------------------------------------------ the whole method

LATTICE_KINDS = {"box": 0, "given": 0, "cbc": 1, "random": 2, "random_smooth": 3}


def _lattice_spec(spec, d):
    """ss_lattice_spec from the pipeline's lattice dictionaries ({"kind": "box",
    "z", "M"}, {"kind": "cbc", "raw", "M_min"}, {"kind": "random", "raw",
    "sigma", "M_min", "smooth"})."""
    kind = spec["kind"]
    if kind == "random" and spec.get("smooth", False):
        kind = "random_smooth"
    ls = LatticeSpec()
    ls.kind = LATTICE_KINDS[kind]
    ls.d = d
    keep = []
    if ls.kind == 0:
        z = np.ascontiguousarray(np.asarray(spec["z"], dtype=np.int64))
        keep.append(z)
        ls.z = z.ctypes.data_as(C.POINTER(C.c_int64))
        ls.M = int(spec["M"])
    else:
        raw = np.ascontiguousarray(np.asarray(spec["raw"], dtype=np.int64))
        keep.append(raw)
        ls.raw = raw.ctypes.data_as(C.POINTER(C.c_int64))
        ls.n_raw = raw.shape[1] if ls.kind == 1 else raw.shape[0]
        ls.M_min = int(spec.get("M_min", 0))
        ls.sigma = float(spec.get("sigma", 0.05))
    ls._keep = keep
    return ls


def sparse_spectral_solve(lattice, a_freq, a_coef, f_freq, f_coef, cand, N, tau=1e-9, sft_precision="fp64",
                          solve_precision="fp64", tol=1e-12, max_iter=1000, raise_on_error=True, out=None):
    """Algorithm 1 in one library call (lattice, SFT of a and f, stamping
    set, right-hand side, solve).  Returns (Stamp, u on S, solve statistics,
    z, M); the caller destroys the stamp.  ``out``: optional complex128
    device tensor; when it holds |S| rows the solution is written into it
    within the call and u is its first |S| rows."""
    cd = _dev_i32(cand)
    d = int(cd.shape[1])
    ls = _lattice_spec(lattice, d)
    a = _trig(a_freq, a_coef, d)
    f = _trig(f_freq, f_coef, d)
    z = (C.c_int64 * d)()
    M = C.c_int64()
    h = C.c_void_p()
    st = SolveStats()
    if out is not None and not (torch.is_tensor(out) and out.is_cuda and out.dtype == torch.complex128
                                and out.is_contiguous()):
        raise TypeError("out must be a contiguous complex128 CUDA tensor")
    cap = out.shape[0] if out is not None else 0
    status = lib.sparse_spectral_solve(C.byref(ls), C.byref(a), C.byref(f), _ptr(cd), cd.shape[0], int(N), float(tau),
                                       _prec(sft_precision), _prec(solve_precision), float(tol), int(max_iter), z,
                                       C.byref(M), C.byref(h), _ptr(out), cap, C.byref(st), _stream())
    if not h.value:
        _check(status if status != 0 else 1)
    stamp = Stamp(h.value, d)
    if status != 0 and raise_on_error:
        msg = lib.ss_last_error().decode(errors="replace")
        stamp.destroy()
        raise SSError(status, msg)
    if out is not None and stamp.size <= cap:
        u = out[: stamp.size]
    else:
        u = torch.empty(stamp.size, dtype=torch.complex128, device="cuda")
        _check(lib.stamp_solution(stamp.handle, _ptr(u), _stream()))
    return stamp, u, st.as_dict(), np.array(z[:], dtype=np.int64), M.value
