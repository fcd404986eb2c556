"""QS^3 hot path on GB300: Python binding of libqs3.so.

Every operation runs in the library's CUDA kernels; this module only
marshals arguments (torch tensors provide device memory and streams).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import QS3_C64, QS3_C128, QS3_C128DF, QS3_C128X, QS3_F32, QS3_F64, QS3Error, check, load

__all__ = ["Basis", "QS3Error", "load", "hphi", "dtype_code", "SolveOpts", "split_df", "probe_peaks",
           "inject_alloc_failure", "inject_wait_timeout"]


def _torch():
    import torch
    return torch


def dtype_code(t) -> int:
    torch = _torch()
    m = {torch.float32: QS3_F32, torch.float64: QS3_F64, torch.complex64: QS3_C64, torch.complex128: QS3_C128}
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return m[t.dtype]


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    if stream is None:
        torch = _torch()
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, n: int | None = None, what: str = "vector"):
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{what} has {t.numel()} elements, expected {n}")
    return ctypes.c_void_p(t.data_ptr())


_PRECISION = {"f64": QS3_F64, "f32": QS3_F32, "df": QS3_C128DF, QS3_F64: QS3_F64, QS3_F32: QS3_F32,
              QS3_C128DF: QS3_C128DF}


class SolveOpts:
    """Fields of qs3_solve_opts with the paper's defaults (input_lancz / input_TRLan).

    precision: "f64" (IEEE binary64 engine), "f32" (fp32 H Phi + binary64
    refinement) or "df" (the double-float engine)."""

    def __init__(self, n_eig=1, n_keep=8, n_max=32, max_iter=10000, min_iter=20, check_every=5, eps=1e-14,
                 precision="f64", use_graphs=True, seed=1, refine_tol=1e-9, res_tol=1e-12, hphi_ieee=False,
                 strict64=False):
        if precision not in _PRECISION:
            raise ValueError(f"precision {precision!r}: use 'f64', 'f32' or 'df'")
        self.n_eig, self.n_keep, self.n_max, self.max_iter = n_eig, n_keep, n_max, max_iter
        self.min_iter, self.check_every, self.eps = min_iter, check_every, eps
        self.precision, self.use_graphs, self.seed, self.refine_tol = precision, use_graphs, seed, refine_tol
        self.res_tol, self.hphi_ieee, self.strict64 = res_tol, hphi_ieee, strict64

    def c(self) -> _abi.qs3_solve_opts:
        o = _abi.qs3_solve_opts()
        o.n_eig, o.n_keep, o.n_max, o.max_iter = self.n_eig, self.n_keep, self.n_max, self.max_iter
        o.min_iter, o.check_every, o.eps = self.min_iter, self.check_every, self.eps
        o.precision = _PRECISION[self.precision]
        o.use_graphs, o.seed, o.refine_tol = int(bool(self.use_graphs)), int(self.seed), float(self.refine_tol)
        o.res_tol = float(self.res_tol)
        o.hphi_ieee = int(bool(self.hphi_ieee))
        o.strict64 = int(bool(self.strict64))
        return o


def split_df(x, out=None, stream=None):
    """Double-float split of a complex128 device vector (qs3_split_df): a
    float32 tensor of 4 x len(x) values (re.hi, re.lo, im.hi, im.lo)."""
    torch = _torch()
    if x.dtype != torch.complex128:
        raise TypeError("x must be complex128")
    if out is None:
        out = torch.empty(4 * x.numel(), dtype=torch.float32, device=x.device)
    check(load().qs3_split_df(_dev(x), _dev(out, 4 * x.numel(), "out"), x.numel(), _stream(stream)), "qs3_split_df")
    return out


def probe_peaks(stream=None) -> dict:
    """Measured throughput of the GPU's arithmetic pipes (qs3_probe_peaks):
    fp64 / fp32 FMA, integer multiply-add and xor/add per second (thread
    operations), warp instructions issued per second and the SM count."""
    p = _abi.qs3_peaks()
    check(load().qs3_probe_peaks(ctypes.byref(p), _stream(stream)), "qs3_probe_peaks")
    return {f: getattr(p, f) for f, _ in p._fields_ if f != "reserved"}


def inject_alloc_failure(after: int) -> int:
    """qs3_inject_alloc_failure: let `after` more device allocations of the
    library succeed and fail every later one with QS3_ERR_OOM (after < 0:
    off).  Returns the previous setting."""
    return int(load().qs3_inject_alloc_failure(int(after)))


def inject_wait_timeout(n: int) -> int:
    """qs3_inject_wait_timeout: the next n copy-ring dot passes launch with
    no copies issued, so their bounded waits run out (QS3_ERR_TIMEOUT);
    n <= 0 switches it off.  Returns the previous count."""
    return int(load().qs3_inject_wait_timeout(int(n)))


def _info_dict(info: _abi.qs3_solve_info) -> dict:
    return {f: getattr(info, f) for f, _ in info._fields_}


class Basis:
    """A set of symmetry sectors (one U(1)-only sector, or several momenta K)
    of one lattice and one number of down spins, built on the device.

    ``lattice`` is any object with n_sites, bi, bj, jxy, jz, h, L (and
    optionally pos) attributes; sites are 0-based.
    """

    def __init__(self, lattice, n_down: int, K=None):
        lib = load()
        self._keep = []

        def arr(a, dt):
            if a is None:
                return None
            x = np.ascontiguousarray(np.asarray(a), dtype=dt)
            self._keep.append(x)
            return x

        lat = _abi.qs3_lattice()
        lat.n_sites = int(lattice.n_sites)
        bi = arr(lattice.bi, np.int32)
        lat.n_bonds = len(bi)
        lat.bi, lat.bj = _ptr(bi), _ptr(arr(lattice.bj, np.int32))
        lat.jxy, lat.jz = _ptr(arr(lattice.jxy, np.float64)), _ptr(arr(lattice.jz, np.float64))
        lat.h = _ptr(arr(getattr(lattice, "h", None), np.float64))
        L = tuple(getattr(lattice, "L", (0, 0, 0)) or (0, 0, 0))
        lat.L[0], lat.L[1], lat.L[2] = int(L[0]), int(L[1]), int(L[2])
        lat.pos = _ptr(arr(getattr(lattice, "pos", None), np.float64))
        lat.n_sub = int(getattr(lattice, "n_sub", 1) or 1)
        self.lattice = lattice
        self.n_down = int(n_down)
        if K is None:
            self.K = None
            nsec, kp = 1, None
        else:
            Ks = [tuple(int(v) for v in k) for k in (K if isinstance(K[0], (tuple, list)) else [K])]
            self.K = Ks
            nsec = len(Ks)
            kp = arr(np.array(Ks, dtype=np.int32).reshape(-1), np.int32)
        h = ctypes.c_void_p()
        check(lib.qs3_basis_create(ctypes.byref(lat), self.n_down, nsec, _ptr(kp), ctypes.byref(h)),
              "qs3_basis_create")
        self._h = h
        n = ctypes.c_int32()
        tot = ctypes.c_uint64()
        check(lib.qs3_basis_info(h, ctypes.byref(n), ctypes.byref(tot)), "qs3_basis_info")
        self.n_sectors = n.value
        self.total_dim = tot.value
        dims = np.zeros(self.n_sectors, np.uint64)
        check(lib.qs3_basis_dims(h, _ptr(dims)), "qs3_basis_dims")
        self.dims = [int(v) for v in dims]
        self.offsets = [0]
        for d in self.dims:
            self.offsets.append(self.offsets[-1] + d)
        self._nnz = None

    @property
    def handle(self):
        return self._h

    @property
    def is_complex(self) -> bool:
        return self.K is not None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().qs3_basis_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ranks(self, s: int = 0):
        """(rank0 array, |Stab| array) of the representatives of sector s."""
        d = self.dims[s]
        r = np.zeros(max(d, 1), np.uint64)
        st = np.zeros(max(d, 1), np.uint8)
        check(load().qs3_basis_ranks(self._h, s, _ptr(r), _ptr(st)), "qs3_basis_ranks")
        return r[:d], st[:d]

    def nnz(self) -> int:
        if self._nnz is None:
            v = ctypes.c_uint64()
            check(load().qs3_basis_nnz(self._h, ctypes.byref(v)), "qs3_basis_nnz")
            self._nnz = v.value
        return self._nnz

    def tuning(self, hphi_blocks_per_sm=None, dot_vectors=None, dot_vectors64=None) -> dict:
        """Autotuned launch choices: query (no arguments) or impose them
        (hphi_blocks_per_sm: up to 5 values indexed by dtype code; 0 = tune again;
        dot_vectors: double-float dot products; dot_vectors64: binary64 ones)."""
        hb = (ctypes.c_int32 * 5)()
        dv = ctypes.c_int32(0)
        dv64 = ctypes.c_int32(0)
        args = (hb, ctypes.byref(dv), ctypes.byref(dv64))
        if hphi_blocks_per_sm is not None or dot_vectors is not None or dot_vectors64 is not None:
            check(load().qs3_basis_tuning(self._h, 0, *args), "qs3_basis_tuning")
            if hphi_blocks_per_sm is not None:
                for i, v in enumerate(hphi_blocks_per_sm):
                    hb[i] = int(v)
            if dot_vectors is not None:
                dv.value = int(dot_vectors)
            if dot_vectors64 is not None:
                dv64.value = int(dot_vectors64)
            check(load().qs3_basis_tuning(self._h, 1, *args), "qs3_basis_tuning")
        check(load().qs3_basis_tuning(self._h, 0, *args), "qs3_basis_tuning")
        return {"hphi_blocks_per_sm": list(hb), "dot_vectors": dv.value, "dot_vectors64": dv64.value}

    def full_diag(self, s: int = 0, vectors: bool = False, stream=None):
        """All eigenvalues (ascending) of sector s, and optionally the eigenvectors
        as the columns of a device complex128 (d, d) tensor."""
        torch = _torch()
        d = self.dims[s]
        ev = np.zeros(max(d, 1), np.float64)
        V = torch.empty((d, d), dtype=torch.complex128, device="cuda") if vectors and d else None
        check(load().qs3_full_diag(self._h, s, _ptr(ev), None if V is None else ctypes.c_void_p(V.data_ptr()),
                                   _stream(stream)), "qs3_full_diag")
        # the library fills column nu contiguously: as a row-major tensor, row nu
        return ev[:d], (None if V is None else V.T)

    def store_terms(self, mode: int = -1) -> int:
        """Stored-term H Phi: 1 build, 0 release, -1 query; returns the device bytes held (0 = off)."""
        v = ctypes.c_uint64()
        check(load().qs3_basis_store_terms(self._h, int(mode), ctypes.byref(v)), "qs3_basis_store_terms")
        return int(v.value)

    def rep_table(self, mode: int = -1) -> bool:
        """Representative table of H Phi: 1 build, 0 release, -1 query; returns whether it is in use."""
        a = ctypes.c_int32()
        check(load().qs3_basis_rep_table(self._h, int(mode), ctypes.byref(a)), "qs3_basis_rep_table")
        return bool(a.value)

    # ---------------------------------------------------------- operations

    def hphi(self, phi, psi=None, stream=None, integer: bool = False):
        """psi = H phi on the device (psi allocated like phi when omitted).
        integer: complex128 only, the binary64 engine's product on the integer
        units (QS3_C128X)."""
        if psi is None:
            psi = _torch().empty_like(phi)
        dt = dtype_code(phi)
        if integer:
            if dt != QS3_C128:
                raise TypeError("the integer product takes complex128 vectors")
            dt = QS3_C128X
        check(load().qs3_hphi(self._h, dt, _dev(phi, self.total_dim, "phi"),
                              _dev(psi, self.total_dim, "psi"), _stream(stream)), "qs3_hphi")
        return psi

    def gs_dots(self, V, w, exact: bool = True, stream=None) -> np.ndarray:
        """conj(V_j) . w per sector (the Gram-Schmidt dots of Alg. 10) as a
        complex (or real) array [n_sectors, m]; V is [m, total_dim] and w
        [total_dim], both float64 or complex128 on the device.  exact: the
        fixed-point exact-accumulation dots of fp64 solves, else binary64
        FMA chains (strict64)."""
        torch = _torch()
        if V.dim() != 2 or V.shape[1] != self.total_dim:
            raise ValueError(f"V must be [m, {self.total_dim}]")
        if V.dtype != w.dtype or V.dtype not in (torch.float64, torch.complex128):
            raise TypeError("V and w must both be float64 or complex128")
        m = int(V.shape[0])
        out = np.zeros((self.n_sectors, m, 2), np.float64)
        check(load().qs3_gs_dots(self._h, dtype_code(V), m, _dev(V), self.total_dim, _dev(w, self.total_dim, "w"),
                                 _ptr(out), 0 if exact else 1, _stream(stream)), "qs3_gs_dots")
        if V.dtype == torch.complex128:
            return out[..., 0] + 1j * out[..., 1]
        return out[..., 0].copy()

    def hphi_df(self, phi_df, psi=None, stream=None):
        """psi = H phi for phi in double-float form (float32 tensor of 4 x the
        total dimension: re.hi, re.lo, im.hi, im.lo per element, see
        split_df); psi is complex128 (allocated when omitted)."""
        torch = _torch()
        if phi_df.dtype != torch.float32:
            raise TypeError("phi_df must be float32 (double-float layout)")
        if psi is None:
            psi = torch.empty(self.total_dim, dtype=torch.complex128, device=phi_df.device)
        if psi.dtype != torch.complex128:
            raise TypeError("psi must be complex128")
        check(load().qs3_hphi(self._h, QS3_C128DF, _dev(phi_df, 4 * self.total_dim, "phi_df"),
                              _dev(psi, self.total_dim, "psi"), _stream(stream)), "qs3_hphi")
        return psi

    def _solve(self, fn, opts: SolveOpts, want_vectors: bool, stream, n_eig: int):
        torch = _torch()
        o = opts.c()
        evals = np.zeros(self.n_sectors * n_eig, np.float64)
        vec = None
        if want_vectors:
            dt = torch.complex128 if self.is_complex else torch.float64
            vec = torch.zeros(n_eig * self.total_dim, dtype=dt, device="cuda")
        info = _abi.qs3_solve_info()
        st = fn(self._h, ctypes.byref(o), _ptr(evals), None if vec is None else _dev(vec), ctypes.byref(info),
                _stream(stream))
        check(st, fn.__name__, allow=(-6,))
        d = _info_dict(info)
        d["status"] = _abi.STATUS.get(st, st)
        return evals.reshape(self.n_sectors, n_eig), vec, d

    def lanczos(self, opts: SolveOpts | None = None, vectors: bool = True, stream=None):
        """Lowest eigenpair per sector: (evals[n_sectors, 1], fp64 vector, info)."""
        return self._solve(load().qs3_lanczos, opts or SolveOpts(), vectors, stream, 1)

    def trlanczos(self, opts: SolveOpts | None = None, vectors: bool = True, stream=None):
        """n_eig lowest eigenpairs per sector by thick-restart Lanczos."""
        opts = opts or SolveOpts()
        return self._solve(load().qs3_trlanczos, opts, vectors, stream, opts.n_eig)

    def correlations(self, gs, sector: int = 0, pairs=None, q=None, local=False, stream=None):
        """Two-point functions and S(q) of the fp64 state gs of one sector."""
        N = int(self.lattice.n_sites)
        pr = None if pairs is None else np.ascontiguousarray(np.asarray(pairs, np.int32).reshape(-1, 2))
        npairs = 0 if pr is None else len(pr)
        qa = None if q is None else np.ascontiguousarray(np.asarray(q, np.float64).reshape(-1, 3))
        nq = 0 if qa is None else len(qa)
        szsz = np.zeros(max(npairs, 1))
        spsm = np.zeros(2 * max(npairs, 1))
        sz = np.zeros(N) if local else None
        sqz = np.zeros(max(nq, 1))
        sqp = np.zeros(max(nq, 1))
        check(load().qs3_correlations(self._h, sector, _dev(gs, self.dims[sector], "gs"), npairs, _ptr(pr),
                                      _ptr(szsz) if npairs else None, _ptr(spsm) if npairs else None, _ptr(sz),
                                      nq, _ptr(qa), _ptr(sqz) if nq else None, _ptr(sqp) if nq else None,
                                      _stream(stream)), "qs3_correlations")
        out = {}
        if npairs:
            out["szsz"] = szsz[:npairs]
            out["spsm"] = spsm[: 2 * npairs].view(np.complex128)
        if local:
            out["sz"] = sz
        if nq:
            out["sq_zz"] = sqz[:nq]
            out["sq_pm"] = sqp[:nq]
        return out


def hphi(basis: Basis, phi, psi=None, stream=None):
    return basis.hphi(phi, psi, stream)


def batch_solve(bases: list, opts: SolveOpts | None = None, max_concurrent: int = 16):
    """Lowest eigenvalue of every sector of many independent bases, solved
    concurrently (qs3_batch_solve).  Returns (list of per-basis eigenvalue
    arrays, list of info dicts, status name)."""
    n = len(bases)
    o = (opts or SolveOpts()).c()
    tot = sum(b.n_sectors for b in bases)
    evals = np.zeros(max(tot, 1), np.float64)
    hs = (ctypes.c_void_p * max(n, 1))(*[b.handle for b in bases])
    infos = (_abi.qs3_solve_info * max(n, 1))()
    st = load().qs3_batch_solve(n, hs, ctypes.byref(o), _ptr(evals), None, infos, int(max_concurrent))
    check(st, "qs3_batch_solve", allow=(-6,))
    out, k = [], 0
    for b in bases:
        out.append(evals[k:k + b.n_sectors].copy())
        k += b.n_sectors
    return out, [_info_dict(infos[i]) for i in range(n)], _abi.STATUS.get(st, st)


def smq(src: Basis, s_src: int, phi, dst: Basis, s_dst: int, Q, psi=None, stream=None):
    """S^-_q phi (Alg. 11, pull form) from sector s_src of src into sector s_dst of dst."""
    torch = _torch()
    if psi is None:
        psi = torch.zeros(dst.dims[s_dst], dtype=torch.complex128, device="cuda")
    q = np.ascontiguousarray(np.asarray(Q, np.int32))
    check(load().qs3_smq(src.handle, s_src, _dev(phi, src.dims[s_src], "phi"), dst.handle, s_dst, _ptr(q),
                         _dev(psi, dst.dims[s_dst], "psi"), _stream(stream)), "qs3_smq")
    return psi


def smq_noalloc(src: Basis, s_src: int, phi, dst: Basis, s_dst: int, Q, psi, stream=None):
    """S^-_q phi without any device allocation during the call (psi must be
    given); asynchronous on the stream."""
    q = np.ascontiguousarray(np.asarray(Q, np.int32))
    check(load().qs3_smq_noalloc(src.handle, s_src, _dev(phi, src.dims[s_src], "phi"), dst.handle, s_dst, _ptr(q),
                                 _dev(psi, dst.dims[s_dst], "psi"), _stream(stream)), "qs3_smq_noalloc")
    return psi


def thermal(E, beta, A=None, mult=None):
    """Eq. (ens) over the levels E: (log Z(beta), <A>(beta)); A = E when None."""
    E = np.ascontiguousarray(E, np.float64)
    b = np.ascontiguousarray(np.atleast_1d(beta), np.float64)
    Aa = None if A is None else np.ascontiguousarray(A, np.float64)
    m = None if mult is None else np.ascontiguousarray(mult, np.float64)
    lz = np.zeros(len(b))
    av = np.zeros(len(b))
    check(load().qs3_thermal(len(E), _ptr(E), _ptr(Aa), _ptr(m), len(b), _ptr(b), _ptr(lz), _ptr(av)), "qs3_thermal")
    return lz, av


OP_SPLUS, OP_SMINUS, OP_SZ = 1, 2, 3


def sq_apply(op: int, src: Basis, s_src: int, phi, dst: Basis, s_dst: int, Q, psi=None, stream=None):
    """S^alpha_q phi (op 1 = S^+, 2 = S^-, 3 = S^z) from sector s_src of src into sector s_dst of dst."""
    if psi is None:
        psi = _torch().zeros(dst.dims[s_dst], dtype=_torch().complex128, device="cuda")
    Qc = np.ascontiguousarray(np.asarray(Q, np.int32).reshape(3))
    check(load().qs3_sq_apply(int(op), src.handle, s_src, _dev(phi, src.dims[s_src], "phi"), dst.handle, s_dst,
                              _ptr(Qc), _dev(psi, dst.dims[s_dst], "psi"), _stream(stream)), "qs3_sq_apply")
    return psi


def dsf(src: Basis, s_src: int, gs, e0: float, dst: Basis, Qs, n_iter: int, eta: float, h_field: float,
        omega: np.ndarray, stream=None, op: int = OP_SMINUS, subtract_trivial: bool = False):
    """S^alpha(q, omega) by the continued fraction for each momentum of Qs
    (dst holds the matching sectors, in order); op 1 = S^+, 2 = S^-, 3 = S^z."""
    Q = np.ascontiguousarray(np.asarray(Qs, np.int32).reshape(-1, 3))
    nq = len(Q)
    om = np.ascontiguousarray(omega, np.float64)
    s = np.zeros(nq * len(om))
    al = np.zeros(nq * n_iter)
    be = np.zeros(nq * n_iter)
    n2 = np.zeros(nq)
    if op == OP_SMINUS and not subtract_trivial:
        check(load().qs3_dsf(src.handle, s_src, _dev(gs, src.dims[s_src], "gs"), float(e0), dst.handle, nq, _ptr(Q),
                             int(n_iter), float(eta), float(h_field), len(om), _ptr(om), _ptr(s), _ptr(al), _ptr(be),
                             _ptr(n2), _stream(stream)), "qs3_dsf")
    else:
        check(load().qs3_dsf_op(int(op), int(bool(subtract_trivial)), src.handle, s_src,
                                _dev(gs, src.dims[s_src], "gs"), float(e0), dst.handle, nq, _ptr(Q), int(n_iter),
                                float(eta), float(h_field), len(om), _ptr(om), _ptr(s), _ptr(al), _ptr(be), _ptr(n2),
                                _stream(stream)), "qs3_dsf_op")
    return s.reshape(nq, len(om)), al.reshape(nq, n_iter), be.reshape(nq, n_iter), n2
