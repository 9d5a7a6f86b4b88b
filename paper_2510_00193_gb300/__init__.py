"""GB300-native Moment Tensor Potential evaluation.

A thin binding over the C-ABI of libmtp_gb300.so (include/mtp.h): every
function here only marshals arguments; neighbour lists, energies, forces,
virials, parameter gradients and grades are computed by the library's CUDA
kernels.  Device arrays are torch tensors on the current CUDA device (torch is
used for device memory and streams only).
"""
from __future__ import annotations

import ctypes
import json

import numpy as np

from . import _lib
from ._lib import MTP_FP64, MTP_GRADE_FP64, MTP_GRADE_TENSOR, MTP_MIXED, MTP_OK, MTP_STATUS_BREAK, MtpError, check

__all__ = [
    "MTP_FP64", "MTP_MIXED", "MTP_GRADE_TENSOR", "MTP_GRADE_FP64", "MtpError", "Potential", "NeighborList", "mtp_basis_info", "mtp_basis_table",
    "mtp_load_params", "mtp_build_neighbors", "mtp_compute_efv", "mtp_compute_efv_noalloc", "mtp_compute_grade",
    "mtp_grade_tc_selftest", "mtp_device_status", "mtp_compute_efv_tangent", "Batch", "mtp_batch_create", "mtp_compute_batch", "mtp_batch_tune",
    "MD", "mtp_compute_basis_rows", "mtp_maxvol", "library_path",
]


def library_path() -> str:
    return _lib.LIB_PATH


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t, dtype=None, n=None, name="array"):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must have dtype %s (got %s)" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if n is not None and t.numel() != n:
        raise ValueError("%s must have %d elements (got %d)" % (name, n, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def _host_d(a, n):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    if a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def mtp_basis_info(level: int) -> dict:
    """Basis size m, radial functions n_mu, moment components, graphs (host only)."""
    lib = _lib.load()
    m, nmu, nc, ng = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    check(lib.mtp_basis_info(level, ctypes.byref(m), ctypes.byref(nmu), ctypes.byref(nc), ctypes.byref(ng)))
    return {"m": m.value, "n_mu": nmu.value, "n_comp": nc.value, "n_graph": ng.value}


def mtp_basis_table(level: int, which: int) -> np.ndarray:
    """Raw int64 table (0 graphs, 1 basis functions, 2 polynomials, 3 components)."""
    lib = _lib.load()
    n = ctypes.c_int64()
    check(lib.mtp_basis_table(level, which, None, ctypes.byref(n)))
    buf = np.zeros(max(1, n.value), dtype=np.int64)
    check(lib.mtp_basis_table(level, which, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(n)))
    return buf[:n.value]


def decode_basis(level: int):
    """(graphs, bases): graphs as (mu tuple, e tuple), bases as tuples of graph indices."""
    g = mtp_basis_table(level, 0).tolist()
    graphs = []
    k = 0
    while k < len(g):
        nv = g[k]
        mu = tuple(g[k + 1:k + 1 + nv])
        ne = nv * (nv - 1) // 2
        e = tuple(g[k + 1 + nv:k + 1 + nv + ne])
        graphs.append((mu, e))
        k += 1 + nv + ne
    b = mtp_basis_table(level, 1).tolist()
    bases = []
    k = 0
    while k < len(b):
        nf = b[k]
        bases.append(tuple(b[k + 1:k + 1 + nf]))
        k += 1 + nf
    return graphs, bases


class Potential:
    """Owns an mtp_handle (parameters resident on the current device)."""

    def __init__(self, level, n_species, n_q, r_min, r_cut, species_energy, radial, xi):
        lib = _lib.load()
        info = mtp_basis_info(level)
        self.level, self.n_species, self.n_q = int(level), int(n_species), int(n_q)
        self.r_min, self.r_cut = float(r_min), float(r_cut)
        self.n_mu = info["n_mu"]
        self.m = info["m"]
        s = _host_d(species_energy, n_species)
        c = _host_d(radial, self.n_mu * n_q * n_species * n_species)
        x = _host_d(xi, len(np.asarray(xi).reshape(-1)))
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
        desc = _lib.ParamsDesc(self.level, self.n_species, self.n_q, self.r_min, self.r_cut, dp(s), dp(c), dp(x),
                               x.size)
        h = ctypes.c_void_p()
        check(lib.mtp_load_params(ctypes.byref(desc), ctypes.byref(h)))
        self._h = h
        n = ctypes.c_int64()
        check(lib.mtp_param_count(h, ctypes.byref(n)))
        self.n_params = n.value
        self._theta0 = np.concatenate([s, c, x])

    def initial_theta(self, device="cuda"):
        """The parameter vector [s | c | xi] the potential was loaded with (FP64 tensor)."""
        import torch
        return torch.tensor(self._theta0, dtype=torch.float64, device=device)

    @classmethod
    def from_dict(cls, pot: dict, check_basis: bool = True):
        """From a potential dictionary (potentials/*.json).  With check_basis the
        file's basis encoding must equal the library's own basis."""
        if check_basis and "basis" in pot:
            graphs, bases = decode_basis(pot["level"])
            mine = [[[list(graphs[k][0]), list(graphs[k][1])] for k in b] for b in bases]
            if mine != pot["basis"]:
                raise ValueError("potential basis differs from the library basis for level %d" % pot["level"])
        return cls(pot["level"], pot["n_species"], pot["n_q"], pot["r_min"], pot["r_cut"], pot["species_energy"],
                   pot["radial"], pot["xi"])

    @classmethod
    def from_file(cls, path: str, check_basis: bool = True):
        with open(path) as fh:
            return cls.from_dict(json.load(fh), check_basis)

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                _lib.load().mtp_free(h)
            except Exception:
                pass
            self._h = None


class NeighborList:
    """Owns an mtp_nlist."""

    def __init__(self):
        self._nl = ctypes.c_void_p()

    @property
    def handle(self):
        return self._nl

    def info(self):
        a, p = ctypes.c_int64(), ctypes.c_int64()
        check(_lib.load().mtp_nlist_info(self._nl, ctypes.byref(a), ctypes.byref(p)))
        return a.value, p.value

    def to_tensors(self, stream=None):
        """(offsets [N+1] int64, j [P] int32, images [P, 3] int32) on the device."""
        import torch
        n, p = self.info()
        dev = torch.device("cuda", torch.cuda.current_device())
        off = torch.empty(n + 1, dtype=torch.int64, device=dev)
        j = torch.empty(max(p, 1), dtype=torch.int32, device=dev)
        img = torch.empty((max(p, 1), 3), dtype=torch.int32, device=dev)
        check(_lib.load().mtp_nlist_copy(self._nl, _dptr(off), _dptr(j), _dptr(img), _stream_ptr(stream)))
        return off, j[:p], img[:p]

    def __del__(self):
        nl = getattr(self, "_nl", None)
        if nl is not None and nl.value:
            try:
                _lib.load().mtp_free_nlist(nl)
            except Exception:
                pass
            self._nl = None


def mtp_load_params(pot: dict) -> Potential:
    return Potential.from_dict(pot)


def mtp_build_neighbors(potential: Potential, x, cell, pbc=(1, 1, 1), nlist: NeighborList | None = None,
                        stream=None) -> NeighborList:
    """Full neighbour list of x ([N, 3] float64 CUDA tensor) in the given cell."""
    import torch
    n = x.shape[0] if x.dim() == 2 else 0
    nl = nlist if nlist is not None else NeighborList()
    c = _host_d(cell, 9)
    p = np.ascontiguousarray(np.asarray(pbc, dtype=np.int32).reshape(3))
    check(_lib.load().mtp_build_neighbors(
        potential.handle, _dptr(x, torch.float64, 3 * n, "x"), n, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(nl.handle), _stream_ptr(stream)))
    return nl


def mtp_compute_efv(potential: Potential, nlist: NeighborList, x, z, cell, precision=MTP_MIXED, chunk_atoms=0,
                    dtheta=False, out=None, stream=None) -> dict:
    """Site energies, forces, virial, total energy and optionally dE/dtheta.

    x: [N, 3] float64, z: [N] int32 (CUDA tensors).  Returns a dict of CUDA
    tensors (e_atom [N], forces [N, 3], virial [6], e_total [1], dtheta or None);
    pass ``out`` (a dict from an earlier call) to reuse its storage."""
    import torch
    n = x.shape[0]
    dev = x.device
    if out is None:
        out = {
            "e_atom": torch.empty(n, dtype=torch.float64, device=dev),
            "forces": torch.empty((n, 3), dtype=torch.float64, device=dev),
            "virial": torch.empty(6, dtype=torch.float64, device=dev),
            "e_total": torch.empty(1, dtype=torch.float64, device=dev),
            "dtheta": torch.empty(potential.n_params, dtype=torch.float64, device=dev) if dtheta else None,
        }
    c = _host_d(cell, 9)
    check(_lib.load().mtp_compute_efv(
        potential.handle, nlist.handle, _dptr(x, torch.float64, 3 * n, "x"), _dptr(z, torch.int32, n, "z"), n,
        c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(precision), int(chunk_atoms),
        _dptr(out["e_atom"], torch.float64, n, "e_atom"), _dptr(out["forces"], torch.float64, 3 * n, "forces"),
        _dptr(out["virial"], torch.float64, 6, "virial"), _dptr(out["e_total"], torch.float64, 1, "e_total"),
        _dptr(out["dtheta"], torch.float64, potential.n_params, "dtheta") if dtheta else None, _stream_ptr(stream)))
    return out


EFV_AUTO, EFV_THREAD_PER_ATOM, EFV_WARP_PER_ATOM = 0, 1, 2


def mtp_set_efv_variant(potential: Potential, variant: int) -> None:
    """Energy/force kernel: 0 tuned/auto, 1 one thread per atom, 2 one warp per atom."""
    check(_lib.load().mtp_set_efv_variant(potential.handle, int(variant)))


def mtp_efv_tune(potential: Potential, nlist: NeighborList, x, z, cell, precision=MTP_MIXED, stream=None) -> dict:
    """Times both energy/force kernels on this configuration and records the
    faster for its size class; returns {"chosen": 1 or 2, "ms": [thread, warp]}."""
    import torch
    n = x.shape[0]
    c = _host_d(cell, 9)
    ch = ctypes.c_int32()
    ms = (ctypes.c_float * 2)()
    check(_lib.load().mtp_efv_tune(potential.handle, nlist.handle, _dptr(x, torch.float64, 3 * n, "x"),
                                   _dptr(z, torch.int32, n, "z"), n, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   int(precision), ctypes.byref(ch), ms, _stream_ptr(stream)))
    return {"chosen": ch.value, "ms": [ms[0], ms[1]]}


def mtp_compute_efv_noalloc(potential: Potential, nlist: NeighborList, x, z, cell, out, chunk_atoms=0,
                            stream=None) -> dict:
    """Mixed-precision site energies, forces, virial and total energy into the
    caller's ``out`` tensors (same keys as mtp_compute_efv), with no device
    allocation inside the library call; at most 65536 atoms."""
    import torch
    n = x.shape[0]
    c = _host_d(cell, 9)
    check(_lib.load().mtp_compute_efv_noalloc(
        potential.handle, nlist.handle, _dptr(x, torch.float64, 3 * n, "x"), _dptr(z, torch.int32, n, "z"), n,
        c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(chunk_atoms),
        _dptr(out["e_atom"], torch.float64, n, "e_atom"), _dptr(out["forces"], torch.float64, 3 * n, "forces"),
        _dptr(out["virial"], torch.float64, 6, "virial"), _dptr(out["e_total"], torch.float64, 1, "e_total"),
        _stream_ptr(stream)))
    return out


def mtp_compute_grade(potential: Potential, nlist: NeighborList, x, z, cell, a_inv=None, a_inv_cfg=None,
                      tau_sel=2.0, tau_brk=10.0, chunk_atoms=0, method=None, out=None, stream=None) -> dict:
    """Extrapolation grades.  a_inv / a_inv_cfg: [m, m] float64 CUDA tensors
    (inverse active sets for neighbourhood / configuration mode).  method:
    MTP_GRADE_TENSOR (default; tensor cores with error-free slicing and an
    FP64 re-check near the thresholds) or MTP_GRADE_FP64.  Returns gamma [N]
    float64 and flags [N] uint8 (CUDA tensors, neighbourhood mode), gamma_max,
    gamma_cfg, n_ambiguous, n_rechecked and status (1 = above the break
    threshold)."""
    import torch
    n = x.shape[0]
    m = potential.m
    dev = x.device
    if method is None:
        method = MTP_GRADE_TENSOR
    if out is None:
        out = {"gamma": torch.empty(n, dtype=torch.float64, device=dev) if a_inv is not None else None,
               "flags": torch.empty(n, dtype=torch.uint8, device=dev) if a_inv is not None else None}
    c = _host_d(cell, 9)
    gmax, gcfg = ctypes.c_double(), ctypes.c_double()
    amb, rchk = ctypes.c_int64(), ctypes.c_int64()
    rc = check(_lib.load().mtp_compute_grade(
        potential.handle, nlist.handle, _dptr(x, torch.float64, 3 * n, "x"), _dptr(z, torch.int32, n, "z"), n,
        c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        _dptr(a_inv, torch.float64, m * m, "a_inv") if a_inv is not None else None,
        _dptr(a_inv_cfg, torch.float64, m * m, "a_inv_cfg") if a_inv_cfg is not None else None,
        float(tau_sel), float(tau_brk), int(chunk_atoms), int(method),
        _dptr(out["gamma"], torch.float64, n, "gamma") if a_inv is not None else None,
        _dptr(out["flags"], torch.uint8, n, "flags") if a_inv is not None else None,
        ctypes.byref(gmax), ctypes.byref(gcfg), ctypes.byref(amb), ctypes.byref(rchk), _stream_ptr(stream)))
    out.update(gamma_max=gmax.value, gamma_cfg=gcfg.value, n_ambiguous=amb.value, n_rechecked=rchk.value, status=rc)
    return out


def mtp_grade_rows(rows, a_inv, tau_sel=2.0, tau_brk=10.0, cols=None, stream=None) -> dict:
    """FP64 grade of the rows of ``rows`` [n, ld] (CUDA float64), restricted
    to the columns ``cols`` (CUDA int32 [m], or all columns), against an
    active-set inverse [m, m]: gamma [n], flags [n], gamma_max, n_ambiguous
    and status (1 = above the break threshold).  With rows = dE/dtheta per
    configuration this is the configuration-mode grade over the parameter
    gradient."""
    import torch
    n, ld = rows.shape
    m = int(cols.numel()) if cols is not None else ld
    gamma = torch.empty(n, dtype=torch.float64, device=rows.device)
    flags = torch.empty(n, dtype=torch.uint8, device=rows.device)
    gmax, amb = ctypes.c_double(), ctypes.c_int64()
    rc = check(_lib.load().mtp_grade_rows(
        _dptr(rows, torch.float64, n * ld, "rows"), int(n), int(ld),
        _dptr(cols, torch.int32, m, "cols") if cols is not None else None, int(m),
        _dptr(a_inv, torch.float64, m * m, "a_inv"), float(tau_sel), float(tau_brk),
        _dptr(gamma, torch.float64, n, "gamma"), _dptr(flags, torch.uint8, n, "flags"), ctypes.byref(gmax),
        ctypes.byref(amb), _stream_ptr(stream)))
    return {"gamma": gamma, "flags": flags, "gamma_max": gmax.value, "n_ambiguous": amb.value, "status": rc}


def mtp_grade_tc_selftest(xs, ys, fexp, erow, n_rows, acc=None, stream=None):
    """Runs the tensor-core grade product on caller-made slices (verification
    hook; layouts as in mtp.h).  xs, ys: int16 CUDA tensors of BF16 bit
    patterns; fexp [128], erow [n_rows]: int32 CUDA tensors; acc: optional
    float32 CUDA tensor [n_rows, 2, 7, 64].  Returns the grades as float64."""
    import torch
    gbits = torch.zeros(n_rows, dtype=torch.int64, device=xs.device)
    tiles = (n_rows + 127) // 128
    check(_lib.load().mtp_grade_tc_selftest(
        _dptr(xs, torch.int16, tiles * 7 * 128 * 128, "xs"), _dptr(ys, torch.int16, 2 * 7 * 64 * 128, "ys"),
        _dptr(fexp, torch.int32, 128, "fexp"), _dptr(erow, torch.int32, n_rows, "erow"), int(n_rows),
        _dptr(acc, torch.float32, n_rows * 2 * 7 * 64, "acc") if acc is not None else None,
        _dptr(gbits, torch.int64, n_rows, "gamma_bits"), _stream_ptr(stream)))
    return gbits.view(torch.float64)


class Batch:
    """Owns an mtp_batch: many small configurations with their neighbour lists."""

    def __init__(self, potential: Potential, atom_off, cells, x, pbc=(1, 1, 1), atoms_per_block=0, stream=None):
        import torch
        lib = _lib.load()
        off = np.ascontiguousarray(np.asarray(atom_off, dtype=np.int64))
        cl = np.ascontiguousarray(np.asarray(cells, dtype=np.float64).reshape(-1))
        p = np.ascontiguousarray(np.asarray(pbc, dtype=np.int32).reshape(3))
        self.n_cfg = len(off) - 1
        self.n_atoms = int(off[-1])
        if cl.size != 9 * self.n_cfg:
            raise ValueError("cells must hold 9 values per configuration")
        self._b = ctypes.c_void_p()
        self._pot = potential
        check(lib.mtp_batch_create(potential.handle, self.n_cfg, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                   cl.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   _dptr(x, torch.float64, 3 * self.n_atoms, "x"), int(atoms_per_block),
                                   ctypes.byref(self._b), _stream_ptr(stream)))

    @property
    def handle(self):
        return self._b

    def nlist_tensors(self, stream=None):
        """(offsets, j, images) of the combined neighbour list."""
        nl = ctypes.c_void_p()
        check(_lib.load().mtp_batch_nlist(self._b, ctypes.byref(nl)))
        view = NeighborList()
        view._nl = nl
        try:
            return view.to_tensors(stream)
        finally:
            view._nl = ctypes.c_void_p()

    def __del__(self):
        b = getattr(self, "_b", None)
        if b is not None and b.value:
            try:
                _lib.load().mtp_batch_free(b)
            except Exception:
                pass
            self._b = None


def _batch_out(potential, batch, x, dtheta):
    import torch
    dev = x.device
    return {"e_cfg": torch.empty(batch.n_cfg, dtype=torch.float64, device=dev),
            "e_atom": torch.empty(batch.n_atoms, dtype=torch.float64, device=dev),
            "forces": torch.empty((batch.n_atoms, 3), dtype=torch.float64, device=dev),
            "virial": torch.empty((batch.n_cfg, 6), dtype=torch.float64, device=dev),
            "dtheta": torch.empty((batch.n_cfg, potential.n_params), dtype=torch.float64, device=dev)
            if dtheta else None}


def mtp_batch_create(potential, atom_off, cells, x, pbc=(1, 1, 1), atoms_per_block=0, stream=None) -> Batch:
    return Batch(potential, atom_off, cells, x, pbc, atoms_per_block, stream)


def mtp_compute_batch(potential: Potential, batch: Batch, x, z, precision=MTP_MIXED, dtheta=False, out=None,
                      stream=None) -> dict:
    """Per-configuration energies e_cfg, per-atom e_atom, forces, per-configuration
    virials and (optionally) dE/dtheta [n_cfg, n_params], as CUDA tensors."""
    import torch
    n = batch.n_atoms
    if out is None:
        out = _batch_out(potential, batch, x, dtheta)
    check(_lib.load().mtp_compute_batch(
        potential.handle, batch.handle, _dptr(x, torch.float64, 3 * n, "x"), _dptr(z, torch.int32, n, "z"),
        int(precision), _dptr(out["e_cfg"], torch.float64, batch.n_cfg, "e_cfg"),
        _dptr(out["e_atom"], torch.float64, n, "e_atom"), _dptr(out["forces"], torch.float64, 3 * n, "forces"),
        _dptr(out["virial"], torch.float64, 6 * batch.n_cfg, "virial"),
        _dptr(out["dtheta"], torch.float64, batch.n_cfg * potential.n_params, "dtheta") if dtheta else None,
        _stream_ptr(stream)))
    return out


def mtp_batch_tune(potential: Potential, batch: Batch, x, z, precision=MTP_MIXED, dtheta=False, stream=None) -> int:
    """Picks the atoms-per-block of the batched launch by timing; returns it."""
    import torch
    out = _batch_out(potential, batch, x, dtheta)
    chosen = ctypes.c_int32()
    n = batch.n_atoms
    check(_lib.load().mtp_batch_tune(
        potential.handle, batch.handle, _dptr(x, torch.float64, 3 * n, "x"), _dptr(z, torch.int32, n, "z"),
        int(precision), int(bool(dtheta)), ctypes.byref(chosen), _dptr(out["e_cfg"]), _dptr(out["forces"]),
        _dptr(out["virial"]), _dptr(out["dtheta"]) if dtheta else None, _stream_ptr(stream)))
    return chosen.value


def mtp_compute_efv_tangent(potential: Potential, nlist: NeighborList, x, z, cell, v, precision=MTP_FP64,
                            force_tan=True, stream=None) -> dict:
    """Directional second derivatives along v ([N, 3] float64 CUDA tensor):
    dtheta_tan = d/dt dE/dtheta (x + t v) and force_tan = d/dt F(x + t v)."""
    import torch
    n = x.shape[0]
    out = {"dtheta_tan": torch.empty(potential.n_params, dtype=torch.float64, device=x.device),
           "force_tan": torch.empty((n, 3), dtype=torch.float64, device=x.device) if force_tan else None}
    c = _host_d(cell, 9)
    check(_lib.load().mtp_compute_efv_tangent(
        potential.handle, nlist.handle, _dptr(x, torch.float64, 3 * n, "x"), _dptr(z, torch.int32, n, "z"), n,
        c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(precision), _dptr(v, torch.float64, 3 * n, "v"),
        _dptr(out["dtheta_tan"], torch.float64, potential.n_params, "dtheta_tan"),
        _dptr(out["force_tan"], torch.float64, 3 * n, "force_tan") if force_tan else None, _stream_ptr(stream)))
    return out


def mtp_set_theta(potential: Potential, theta, stream=None) -> None:
    """Replace the potential's parameters by theta (CUDA FP64 tensor
    [n_params], layout [s | c | xi]); queued on ``stream``."""
    import torch
    check(_lib.load().mtp_set_theta(potential.handle, _dptr(theta, torch.float64, potential.n_params, "theta"),
                                    _stream_ptr(stream)))


def mtp_device_status(potential: Potential, stream=None) -> int:
    """Device-side status since the last check (0 = fine); raises on error."""
    return check(_lib.load().mtp_device_status(potential.handle, _stream_ptr(stream)))


def mtp_compute_basis_rows(potential: Potential, nlist: NeighborList, x, z, cell, out=None, stream=None):
    """FP64 basis rows [N, m] (CUDA tensor) of every atom."""
    import torch
    n = x.shape[0]
    if out is None:
        out = torch.empty((n, potential.m), dtype=torch.float64, device=x.device)
    c = _host_d(cell, 9)
    check(_lib.load().mtp_compute_basis_rows(
        potential.handle, nlist.handle, _dptr(x, torch.float64, 3 * n, "x"), _dptr(z, torch.int32, n, "z"), n,
        c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _dptr(out, torch.float64, n * potential.m, "rows"),
        _stream_ptr(stream)))
    return out


def mtp_maxvol(pool, rows, delta=0.01, max_iter=10000, stream=None):
    """MaxVol active set of pool ([n_pool, m] float64 CUDA tensor) from the
    initial rows; returns (rows as an int32 numpy array, A^-1 [m, m] CUDA
    tensor, number of swaps)."""
    import torch
    n, m = pool.shape
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int32).reshape(-1)).copy()
    if r.size != m:
        raise ValueError("rows must hold m = %d indices" % m)
    a_inv = torch.empty((m, m), dtype=torch.float64, device=pool.device)
    it = ctypes.c_int32()
    check(_lib.load().mtp_maxvol(_dptr(pool, torch.float64, n * m, "pool"), n, m,
                                 r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), float(delta), int(max_iter),
                                 _dptr(a_inv, torch.float64, m * m, "a_inv"), ctypes.byref(it), _stream_ptr(stream)))
    return r, a_inv, it.value


class MD:
    """Owns an mtp_md: velocity-Verlet molecular dynamics with a skin
    neighbour list filtered to the exact list every step (include/mtp.h)."""

    def __init__(self, potential: Potential, x, cell, pbc=(1, 1, 1), skin=0.3, stream=None):
        import torch
        n = x.shape[0]
        c = _host_d(cell, 9)
        p = np.ascontiguousarray(np.asarray(pbc, dtype=np.int32).reshape(3))
        self.n_atoms = n
        self.cell = c
        self._pot = potential
        self._md = ctypes.c_void_p()
        check(_lib.load().mtp_md_create(
            potential.handle, _dptr(x, torch.float64, 3 * n, "x"), n, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), float(skin), ctypes.byref(self._md), _stream_ptr(stream)))

    @property
    def handle(self):
        return self._md

    def rebuild(self, x, stream=None):
        import torch
        check(_lib.load().mtp_md_rebuild(self._pot.handle, self._md, _dptr(x, torch.float64, 3 * self.n_atoms, "x"),
                                         _stream_ptr(stream)))

    def nlist(self, stream=None) -> NeighborList:
        """The exact list of the current positions (a view owned by this object)."""
        nl = ctypes.c_void_p()
        check(_lib.load().mtp_md_nlist(self._md, ctypes.byref(nl), _stream_ptr(stream)))
        view = _NeighborListView()
        view._nl = nl
        view._owner = self
        return view

    def status(self, stream=None) -> int:
        """Steps run on the current skin list; raises MtpError (MTP_ERR_STALE_LIST)
        if an atom moved more than skin/2 since its build."""
        k = ctypes.c_int64()
        check(_lib.load().mtp_md_status(self._md, ctypes.byref(k), None, _stream_ptr(stream)))
        return k.value

    def rebuilds(self, stream=None) -> int:
        """Skin-list builds since creation (the first included)."""
        k = ctypes.c_int64()
        check(_lib.load().mtp_md_status(self._md, None, ctypes.byref(k), _stream_ptr(stream)))
        return k.value

    def run(self, x, v, z, masses, dt, n_steps, forces, rebuild_every=0, precision=MTP_MIXED, e_pot=None, e_kin=None,
            stream=None):
        """n_steps velocity-Verlet steps in place on x, v and forces (CUDA
        tensors [N, 3] float64; forces must hold the forces at x on entry).
        masses: per species, amu; dt in ps.  rebuild_every: < 0 check the
        displacements every step and rebuild when needed, > 0 rebuild every
        that many steps, 0 never (no synchronisation).  e_pot / e_kin: optional
        CUDA tensors [n_steps] float64 that receive the energies after each step.
        Returns MTP_OK, or MTP_STATUS_BREAK when an in-run grade (set_grade)
        exceeded the break threshold (the run stopped after that step)."""
        import torch
        n = self.n_atoms
        m = _host_d(masses, self._pot.n_species)
        return check(_lib.load().mtp_md_run(
            self._pot.handle, self._md, _dptr(x, torch.float64, 3 * n, "x"), _dptr(v, torch.float64, 3 * n, "v"),
            _dptr(z, torch.int32, n, "z"), m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(dt), int(n_steps),
            int(rebuild_every), int(precision), _dptr(forces, torch.float64, 3 * n, "forces"),
            _dptr(e_pot, torch.float64, n_steps, "e_pot") if e_pot is not None else None,
            _dptr(e_kin, torch.float64, n_steps, "e_kin") if e_kin is not None else None, _stream_ptr(stream)))

    def set_grade(self, a_inv, every, tau_sel=2.0, tau_brk=10.0, method=MTP_GRADE_TENSOR, selected=None):
        """Evaluate the neighbourhood grade every ``every`` steps inside run();
        ``selected`` (CUDA uint8 [N], optional) accumulates the flags.  a_inv=None turns it off."""
        import torch
        m = self._pot.m
        self._a_inv = a_inv   # kept alive: the library holds the pointer
        self._selected = selected
        check(_lib.load().mtp_md_set_grade(
            self._pot.handle, self._md, _dptr(a_inv, torch.float64, m * m, "a_inv") if a_inv is not None else None,
            int(every), float(tau_sel), float(tau_brk), int(method),
            _dptr(selected, torch.uint8, self.n_atoms, "selected") if selected is not None else None))

    def set_barostat(self, p_target_bar, tau_p_ps, bulk_modulus_bar=10.0):
        """Berendsen NPT (isotropic); tau_p_ps <= 0 turns it off."""
        check(_lib.load().mtp_md_set_barostat(self._md, float(p_target_bar), float(tau_p_ps), float(bulk_modulus_bar)))

    def info(self) -> dict:
        st, ev, ns = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        gm, pr = ctypes.c_double(), ctypes.c_double()
        cell = np.zeros(9)
        check(_lib.load().mtp_md_info(self._md, ctypes.byref(st), ctypes.byref(ev), ctypes.byref(gm), ctypes.byref(ns),
                                      ctypes.byref(pr), cell.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return {"steps": st.value, "grade_evals": ev.value, "gamma_max_last": gm.value,
                "n_selected_last": ns.value, "pressure_bar": pr.value, "cell": cell.reshape(3, 3)}

    def __del__(self):
        md = getattr(self, "_md", None)
        if md is not None and md.value:
            try:
                _lib.load().mtp_md_free(md)
            except Exception:
                pass
            self._md = None


class _NeighborListView(NeighborList):
    """A neighbour list owned by another object (not freed here)."""

    def __del__(self):
        self._nl = None


PROBE_FP32, PROBE_FP64, PROBE_FP32X2 = 0, 1, 2


def mtp_probe_fma(kind=PROBE_FP32, iters=4096, blocks_per_sm=4) -> dict:
    """Measured FMA throughput of the current device (flop/s and the timed
    kernel's ms): kind 0 FP32, 1 FP64, 2 packed FP32 pairs."""
    f = ctypes.c_double()
    ms = ctypes.c_double()
    check(_lib.load().mtp_probe_fma(int(kind), int(iters), int(blocks_per_sm), ctypes.byref(f), ctypes.byref(ms)))
    return {"flops_per_s": f.value, "ms": ms.value}
