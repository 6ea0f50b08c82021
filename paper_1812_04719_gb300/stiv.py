"""Python binding of libstiv (the C-ABI in include/stiv.h).

Argument marshalling only: every step of the path runs in the CUDA kernels of
libstiv.so.  PyTorch supplies device memory and streams.  If the library is
missing this module raises at import time of ``lib()``; there is no CPU path.

Low level: ``stiv_create``, ``stiv_upsample``, ``stiv_detect``, ``stiv_stiv``,
``stiv_stiv_grad``, ``stiv_grad_scatter``, ``stiv_grad_to_coef``, ``stiv_step``,
``stiv_sync_counts``, ``stiv_mesh_topology``, ``stiv_sort_pairs`` take raw
device pointers (ints) like the C functions.  High level: ``Stiv`` runs the
per-step path of Alg. 2 (upsample, detect, volumes and gradient) on a scene
held in device tensors and grows its output buffers when the kernels report
an overflow.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstiv.so")

STIV_OK, STIV_ERR_ARG, STIV_ERR_CAPACITY, STIV_ERR_TIMEOUT, STIV_ERR_CUDA, STIV_ERR_INPUT = range(6)
STIV_FP64, STIV_MIXED = 0, 1
STIV_VEL_RELATIVE, STIV_VEL_ABSOLUTE = 0, 1
C_PAIRS, C_PRIM, C_VF, C_EE, C_CPAIRS, C_DEGEN, C_STATUS, C_PATCH, C_FLOPS, C_EXACT, C_PIECE = range(11)
NCOUNTS = 11
F_PAIRS_OVERFLOW, F_CONTACTS_OVERFLOW, F_BOX_TOO_SMALL, F_NONFINITE, F_WORK_OVERFLOW, F_TIMEOUT = 1, 2, 4, 8, 16, 32
F_BAD_ORDER = 64
MAX_ORDER = 32   # largest SH order p the library accepts (mesh order 64)

EXPORTS = ["stiv_create", "stiv_destroy", "stiv_status_string", "stiv_last_cuda_error", "stiv_mesh_topology",
           "stiv_upsample", "stiv_detect", "stiv_stiv", "stiv_stiv_grad", "stiv_grad_scatter",
           "stiv_grad_to_coef", "stiv_step", "stiv_sync_counts", "stiv_sort_scratch_bytes", "stiv_sort_pairs",
           "stiv_profile", "stiv_profile_read", "stiv_sort_pairs_static", "stiv_autotune", "stiv_set_tuning",
           "stiv_wait_selftest", "stiv_lcp_matrix", "stiv_lcp_solve",
           "stiv_mesh_fidelity", "stiv_stiv_grad_x0", "stiv_peak_probe"]
TUNE_NAMES = ("narrow_ctas_per_sm", "pieces_ctas_per_sm", "fp64_blocks_per_sm", "patch_blocks_per_sm",
              "piece_levels")
SORT_STATIC_MAX = 1 << 20


class StivError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})" if what else status_string(status))


class StivLcp(ctypes.Structure):
    _fields_ = [("row_capacity", ctypes.c_int64), ("nnz_capacity", ctypes.c_int64), ("row_pair", ctypes.c_void_p),
                ("q", ctypes.c_void_p), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("dims", ctypes.c_void_p)]


class StivParams(ctypes.Structure):
    _fields_ = [("d_m", ctypes.c_double), ("eps", ctypes.c_double), ("dt", ctypes.c_double),
                ("box_L", ctypes.c_double * 3), ("precision", ctypes.c_int32), ("include_ee", ctypes.c_int32),
                ("exact_only", ctypes.c_int32), ("velocity", ctypes.c_int32)]


class StivPairs(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("i", ctypes.c_void_p), ("j", ctypes.c_void_p),
                ("shift", ctypes.c_void_p)]


class StivContacts(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("pair", ctypes.c_void_p), ("type", ctypes.c_void_p),
                ("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("tau", ctypes.c_void_p), ("w", ctypes.c_void_p)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libstiv.so (built by ``paper_1812_04719_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libstiv.so not found at {LIB_PATH}: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER
    L.stiv_create.argtypes = [P(vp), P(StivParams)]
    L.stiv_destroy.argtypes = [vp]
    L.stiv_status_string.argtypes = [ctypes.c_int]
    L.stiv_status_string.restype = ctypes.c_char_p
    L.stiv_last_cuda_error.argtypes = [vp]
    L.stiv_mesh_topology.argtypes = [i32, vp, vp, vp]
    L.stiv_upsample.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp]
    L.stiv_detect.argtypes = [vp, vp, i32, i32, vp, vp, vp, P(StivPairs), P(StivContacts), vp]
    L.stiv_stiv.argtypes = [vp, vp, i32, vp, vp, vp, P(StivPairs), P(StivContacts), vp, vp, vp]
    L.stiv_stiv_grad.argtypes = [vp, vp, i32, vp, vp, vp, P(StivPairs), P(StivContacts), vp, vp, vp, vp, vp, vp]
    L.stiv_grad_scatter.argtypes = [vp, vp, vp, P(StivContacts), vp, vp, vp, vp, vp, vp, vp]
    L.stiv_grad_to_coef.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp]
    L.stiv_step.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, vp, vp, P(StivPairs), P(StivContacts), vp, vp, vp,
                            vp, vp, vp]
    L.stiv_sync_counts.argtypes = [vp, vp, vp]
    L.stiv_sort_scratch_bytes.argtypes = [i64]
    L.stiv_sort_scratch_bytes.restype = ctypes.c_size_t
    L.stiv_sort_pairs.argtypes = [vp, i64, i32, vp, vp, vp, vp, vp, ctypes.c_size_t]
    L.stiv_sort_pairs_static.argtypes = [vp, i64, i32, vp, vp, vp, vp]
    L.stiv_autotune.argtypes = [vp, vp, i32, i32, vp, vp, vp, P(StivPairs), P(StivContacts), vp, vp, vp]
    L.stiv_set_tuning.argtypes = [vp, vp]
    L.stiv_wait_selftest.argtypes = [vp, i64, vp]
    L.stiv_lcp_matrix.argtypes = [vp, vp, i32, i32, P(StivPairs), P(StivContacts), vp, vp, vp, vp, vp, vp, vp,
                                  P(StivLcp)]
    L.stiv_stiv_grad_x0.argtypes = [vp, vp, i32, vp, vp, vp, P(StivPairs), P(StivContacts), vp, vp]
    L.stiv_mesh_fidelity.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp, i32, vp]
    L.stiv_lcp_solve.argtypes = [vp, vp, P(StivLcp), ctypes.c_double, i32, i32, vp, vp]
    L.stiv_peak_probe.argtypes = [vp, i32, i64, vp, P(ctypes.c_double)]
    L.stiv_profile.argtypes = [vp, i32]
    L.stiv_profile_read.argtypes = [vp, i32, vp, vp, vp, vp]
    _lib = L
    return L


def status_string(s: int) -> str:
    try:
        return lib().stiv_status_string(int(s)).decode()
    except Exception:
        return f"status {s}"


def _check(rc: int, what: str):
    if rc != STIV_OK:
        raise StivError(rc, what)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


# ---------------------------------------------------------------------------
# low-level: same names as the C entry points, raw pointers
# ---------------------------------------------------------------------------

def stiv_create(d_m=0.0, eps=1.0, dt=0.1, box_L=(0.0, 0.0, 0.0), precision=STIV_FP64, include_ee=True,
                exact_only=False, velocity=0) -> int:
    prm = StivParams(float(d_m), float(eps), float(dt), (ctypes.c_double * 3)(*[float(x) for x in box_L]),
                     int(precision), int(bool(include_ee)), int(bool(exact_only)), int(velocity))
    h = ctypes.c_void_p()
    _check(lib().stiv_create(ctypes.byref(h), ctypes.byref(prm)), "stiv_create")
    return h.value


def stiv_destroy(h: int):
    _check(lib().stiv_destroy(h), "stiv_destroy")


def stiv_mesh_topology(P: int, tri_ptr: int, edge_ptr: int, stream: int):
    _check(lib().stiv_mesh_topology(P, tri_ptr, edge_ptr, stream), "stiv_mesh_topology")


def stiv_upsample(h, stream, n_ves, p_max, p_ptr, coef_off_ptr, coef_ptr, vert_off_ptr, verts_ptr):
    _check(lib().stiv_upsample(h, stream, n_ves, p_max, p_ptr, coef_off_ptr, coef_ptr, vert_off_ptr, verts_ptr),
           "stiv_upsample")


def stiv_detect(h, stream, n_ves, p_max, p_ptr, vert_off_ptr, verts_ptr, cand: StivPairs, out: StivContacts,
                counts_ptr):
    _check(lib().stiv_detect(h, stream, n_ves, p_max, p_ptr, vert_off_ptr, verts_ptr, ctypes.byref(cand),
                             ctypes.byref(out), counts_ptr), "stiv_detect")


def stiv_stiv(h, stream, n_ves, p_ptr, vert_off_ptr, verts_ptr, cand, contacts, counts_ptr, Vc_ptr, Vp_ptr):
    _check(lib().stiv_stiv(h, stream, n_ves, p_ptr, vert_off_ptr, verts_ptr, ctypes.byref(cand),
                           ctypes.byref(contacts), counts_ptr, Vc_ptr, Vp_ptr), "stiv_stiv")


def stiv_stiv_grad(h, stream, n_ves, p_ptr, vert_off_ptr, verts_ptr, cand, contacts, counts_ptr, Vc_ptr, Vp_ptr,
                   grad_ptr, gves_ptr, gvid_ptr):
    _check(lib().stiv_stiv_grad(h, stream, n_ves, p_ptr, vert_off_ptr, verts_ptr, ctypes.byref(cand),
                                ctypes.byref(contacts), counts_ptr, Vc_ptr, Vp_ptr, grad_ptr, gves_ptr, gvid_ptr),
           "stiv_stiv_grad")


def stiv_grad_scatter(h, stream, p_ptr, contacts, counts_ptr, wpair_ptr, grad_ptr, gves_ptr, gvid_ptr,
                      vert_off_ptr, gX_ptr):
    _check(lib().stiv_grad_scatter(h, stream, p_ptr, ctypes.byref(contacts), counts_ptr, wpair_ptr, grad_ptr,
                                   gves_ptr, gvid_ptr, vert_off_ptr, gX_ptr), "stiv_grad_scatter")


def stiv_grad_to_coef(h, stream, n_ves, p_max, p_ptr, coef_off_ptr, vert_off_ptr, gX_ptr, gcoef_ptr):
    _check(lib().stiv_grad_to_coef(h, stream, n_ves, p_max, p_ptr, coef_off_ptr, vert_off_ptr, gX_ptr, gcoef_ptr),
           "stiv_grad_to_coef")


def stiv_step(h, stream, use_graph, n_ves, p_max, p_ptr, coef_off_ptr, coef_ptr, vert_off_ptr, verts_ptr, cand,
              out, counts_ptr, Vc_ptr, Vp_ptr, grad_ptr, gves_ptr, gvid_ptr):
    _check(lib().stiv_step(h, stream, int(use_graph), n_ves, p_max, p_ptr, coef_off_ptr, coef_ptr, vert_off_ptr,
                           verts_ptr, ctypes.byref(cand), ctypes.byref(out), counts_ptr, Vc_ptr, Vp_ptr, grad_ptr,
                           gves_ptr, gvid_ptr), "stiv_step")


def stiv_sync_counts(stream, counts_ptr):
    host = np.zeros(NCOUNTS, dtype=np.int64)
    rc = lib().stiv_sync_counts(stream, counts_ptr, host.ctypes.data)
    return rc, host


def stiv_sort_pairs(stream, n, key_bits, keys_in_ptr, vals_in_ptr, keys_out_ptr, vals_out_ptr, scratch_ptr,
                    scratch_bytes):
    _check(lib().stiv_sort_pairs(stream, n, key_bits, keys_in_ptr, vals_in_ptr, keys_out_ptr, vals_out_ptr,
                                 scratch_ptr, scratch_bytes), "stiv_sort_pairs")


def stiv_sort_pairs_static(stream, n, key_bits, keys_in_ptr, vals_in_ptr, keys_out_ptr, vals_out_ptr):
    """Same sort as stiv_sort_pairs without caller scratch: it runs on a fixed
    static device array of the library (n <= SORT_STATIC_MAX).  For callers
    that cannot allocate device memory; calls that overlap on the GPU race."""
    _check(lib().stiv_sort_pairs_static(stream, n, key_bits, keys_in_ptr, vals_in_ptr, keys_out_ptr,
                                        vals_out_ptr), "stiv_sort_pairs_static")


def stiv_peak_probe(stream, kind: int, iters: int, sink_ptr: int) -> float:
    """Launch the FMA-rate probe (kind 0 FP64, 1 FP32); returns the FLOPs the
    launch performs (time it with events on the same stream)."""
    fl = ctypes.c_double(0.0)
    _check(lib().stiv_peak_probe(stream, int(kind), int(iters), sink_ptr, ctypes.byref(fl)), "stiv_peak_probe")
    return fl.value


def stiv_profile(h: int, enable: bool):
    _check(lib().stiv_profile(h, int(bool(enable))), "stiv_profile")


def stiv_profile_read(h: int) -> dict:
    """{stage: (launches, total_ms)} since the last read."""
    maxn = 64
    names = ctypes.create_string_buffer(32 * maxn)
    cnt = np.zeros(maxn, dtype=np.int64)
    tot = np.zeros(maxn, dtype=np.float64)
    n = ctypes.c_int32(0)
    _check(lib().stiv_profile_read(h, maxn, ctypes.addressof(names), cnt.ctypes.data, tot.ctypes.data,
                                   ctypes.addressof(n)), "stiv_profile_read")
    out = {}
    for k in range(min(n.value, maxn)):
        nm = names.raw[32 * k:32 * k + 32].split(b"\0", 1)[0].decode()
        out[nm] = (int(cnt[k]), float(tot[k]))
    return out


def stiv_sort_scratch_bytes(n: int) -> int:
    return int(lib().stiv_sort_scratch_bytes(int(n)))


# ---------------------------------------------------------------------------
# high level
# ---------------------------------------------------------------------------

def nverts(P: int) -> int:
    return 2 * P * (P + 1) + 2


@dataclass
class DeviceScene:
    """Scene inputs resident on the device, in the library's layouts."""
    n: int
    p_max: int
    p: torch.Tensor          # int32 [N]
    coef_off: torch.Tensor   # int64 [N]
    coef: torch.Tensor       # float64 flat
    vert_off: torch.Tensor   # int64 [N]
    verts: torch.Tensor      # float64 or float32 flat
    box_L: tuple
    eps: float
    dt: float
    d_m: float

    @staticmethod
    def from_scene(sc, precision=STIV_FP64, device="cuda") -> "DeviceScene":
        dt = torch.float32 if precision == STIV_MIXED else torch.float64
        p = np.asarray(sc.p)
        if p.size and (p.min() < 1 or p.max() > MAX_ORDER):
            raise ValueError(f"SH orders must lie in [1, {MAX_ORDER}], got [{p.min()}, {p.max()}]")
        vo = sc.vert_off()
        return DeviceScene(
            n=sc.n, p_max=int(sc.p.max()),
            p=torch.as_tensor(sc.p, dtype=torch.int32, device=device),
            coef_off=torch.as_tensor(sc.coef_off, dtype=torch.int64, device=device),
            coef=torch.as_tensor(sc.coef, dtype=torch.float64, device=device),
            vert_off=torch.as_tensor(vo, dtype=torch.int64, device=device),
            verts=torch.zeros(sc.n_vert_values(), dtype=dt, device=device),
            box_L=tuple(float(x) for x in sc.L), eps=float(sc.eps), dt=float(sc.dt), d_m=float(sc.d_m))


class Buffers:
    """Output buffers of one step, sized by capacities."""

    def __init__(self, device, pair_cap: int, contact_cap: int, grad: bool):
        self.pair_cap, self.contact_cap = int(pair_cap), int(contact_cap)
        i32 = dict(dtype=torch.int32, device=device)
        f64 = dict(dtype=torch.float64, device=device)
        self.ci = torch.zeros(self.pair_cap, **i32)
        self.cj = torch.zeros(self.pair_cap, **i32)
        self.cs = torch.zeros(self.pair_cap, **i32)
        self.pair = torch.zeros(self.contact_cap, **i32)
        self.type = torch.zeros(self.contact_cap, **i32)
        self.a = torch.zeros(self.contact_cap, **i32)
        self.b = torch.zeros(self.contact_cap, **i32)
        self.tau = torch.zeros(self.contact_cap, **f64)
        self.w = torch.zeros(self.contact_cap, 2, **f64)
        self.counts = torch.zeros(NCOUNTS, dtype=torch.int64, device=device)
        self.Vc = torch.zeros(self.contact_cap, **f64)
        self.Vp = torch.zeros(self.pair_cap, **f64)
        self.grad = torch.zeros(self.contact_cap, 4, 3, **f64) if grad else None
        self.gves = torch.zeros(self.contact_cap, 4, **i32) if grad else None
        self.gvid = torch.zeros(self.contact_cap, 4, **i32) if grad else None

    def pairs_struct(self) -> StivPairs:
        return StivPairs(self.pair_cap, _ptr(self.ci), _ptr(self.cj), _ptr(self.cs))

    def contacts_struct(self) -> StivContacts:
        return StivContacts(self.contact_cap, _ptr(self.pair), _ptr(self.type), _ptr(self.a), _ptr(self.b),
                            _ptr(self.tau), _ptr(self.w))


class Stiv:
    """One library handle plus the buffers of the per-step path."""

    def __init__(self, box_L=(0.0, 0.0, 0.0), eps=1.0, dt=0.1, d_m=0.0, precision=STIV_FP64, include_ee=True,
                 pair_cap=1024, contact_cap=1 << 16, device="cuda", exact_only=False, velocity=STIV_VEL_RELATIVE):
        self.precision = precision
        self.device = torch.device(device)
        self.h = stiv_create(d_m=d_m, eps=eps, dt=dt, box_L=box_L, precision=precision, include_ee=include_ee,
                             exact_only=exact_only, velocity=velocity)
        self.pair_cap, self.contact_cap = pair_cap, contact_cap
        self.buf = None

    @staticmethod
    def for_scene(sc, precision=STIV_FP64, **kw) -> "Stiv":
        return Stiv(box_L=tuple(sc.L), eps=sc.eps, dt=sc.dt, d_m=sc.d_m, precision=precision, **kw)

    def close(self):
        if self.h:
            stiv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _buffers(self, grad: bool) -> Buffers:
        b = self.buf
        if b is None or b.pair_cap != self.pair_cap or b.contact_cap != self.contact_cap or (grad and b.grad is None):
            self.buf = Buffers(self.device, self.pair_cap, self.contact_cap, grad)
        return self.buf

    def upsample(self, ds: DeviceScene, stream=None):
        stiv_upsample(self.h, _stream(stream), ds.n, ds.p_max, _ptr(ds.p), _ptr(ds.coef_off), _ptr(ds.coef),
                      _ptr(ds.vert_off), _ptr(ds.verts))

    def step(self, ds: DeviceScene, grad: bool = True, upsample: bool = True, use_graph: bool = False,
             stream=None, max_retries: int = 8) -> dict:
        """upsample (optional) + detect + V (+ dV/dX1).  Returns host counts and
        device views of the outputs trimmed to their counts."""
        st = _stream(stream)
        for _ in range(max_retries):
            b = self._buffers(grad)
            cand, out = b.pairs_struct(), b.contacts_struct()
            # coef NULL: ds.verts is the input, the upsampling is skipped
            stiv_step(self.h, st, use_graph, ds.n, ds.p_max, _ptr(ds.p), _ptr(ds.coef_off),
                      _ptr(ds.coef) if upsample else 0, _ptr(ds.vert_off), _ptr(ds.verts), cand, out, _ptr(b.counts),
                      _ptr(b.Vc), _ptr(b.Vp), _ptr(b.grad) if grad else 0, _ptr(b.gves) if grad else 0,
                      _ptr(b.gvid) if grad else 0)
            rc, counts = stiv_sync_counts(st, _ptr(b.counts))
            if rc == STIV_ERR_CAPACITY:
                f = int(counts[C_STATUS])
                if f & F_PAIRS_OVERFLOW or f & F_WORK_OVERFLOW:
                    self.pair_cap = max(2 * self.pair_cap, int(counts[C_PAIRS]) + 16)
                if f & F_CONTACTS_OVERFLOW or f & F_WORK_OVERFLOW:
                    self.contact_cap = max(2 * self.contact_cap, int(counts[C_VF] + counts[C_EE]) + 16)
                continue
            _check(rc, "step")
            return self.result(counts, grad)
        raise StivError(STIV_ERR_CAPACITY, "step: capacities kept overflowing")

    def autotune(self, ds: DeviceScene, stream=None, max_retries: int = 8) -> dict:
        """Pick the narrow phase's launch shapes for this workload (the
        library times its detection under candidates and keeps the fastest).
        Returns {parameter: value, "best_ms": detection time}."""
        st = _stream(stream)
        self.step(ds, grad=False, stream=stream)      # upsampled vertices and sized buffers
        choice = np.zeros(len(TUNE_NAMES), dtype=np.int32)
        best = ctypes.c_double(0.0)
        for _ in range(max_retries):
            b = self._buffers(False)
            cand, out = b.pairs_struct(), b.contacts_struct()
            rc = lib().stiv_autotune(self.h, st, ds.n, ds.p_max, _ptr(ds.p), _ptr(ds.vert_off), _ptr(ds.verts),
                                     ctypes.byref(cand), ctypes.byref(out), _ptr(b.counts), choice.ctypes.data,
                                     ctypes.addressof(best))
            if rc == STIV_ERR_CAPACITY:
                self.step(ds, grad=False, stream=stream)   # grows the capacities
                continue
            _check(rc, "stiv_autotune")
            res = {k: int(v) for k, v in zip(TUNE_NAMES, choice)}
            res["best_ms"] = best.value
            return res
        raise StivError(STIV_ERR_CAPACITY, "autotune: capacities kept overflowing")

    def grad_x0(self, ds: DeviceScene, stream=None) -> torch.Tensor:
        """dV_k/dX0 rows [contacts][4][3] of the last step's contacts (points
        as in that step's gves / gvid)."""
        b = self.buf
        nc = int(b.counts[C_VF].item() + b.counts[C_EE].item())
        g0 = torch.zeros(max(b.contact_cap, 1), 4, 3, dtype=torch.float64, device=self.device)
        _check(lib().stiv_stiv_grad_x0(self.h, _stream(stream), ds.n, _ptr(ds.p), _ptr(ds.vert_off), _ptr(ds.verts),
                                       ctypes.byref(b.pairs_struct()), ctypes.byref(b.contacts_struct()),
                                       _ptr(b.counts), _ptr(g0)), "stiv_stiv_grad_x0")
        return g0[:nc]

    def mesh_fidelity(self, ds: DeviceScene, factor: int = 4, stream=None) -> torch.Tensor:
        """Per vesicle and time level, the largest distance between the order-2p
        triangle mesh in ds.verts (as upsampled) and the smooth order-p surface,
        on the order-(factor 2p) grid (Sec. 3.1.2, Fig. 6).  float64 [n, 2]."""
        err = torch.zeros(ds.n, 2, dtype=torch.float64, device=self.device)
        _check(lib().stiv_mesh_fidelity(self.h, _stream(stream), ds.n, ds.p_max, _ptr(ds.p), _ptr(ds.coef_off),
                                        _ptr(ds.coef), _ptr(ds.vert_off), _ptr(ds.verts), int(factor), _ptr(err)),
               "stiv_mesh_fidelity")
        return err

    def set_tuning(self, **values):
        """Pin launch shapes by name (see TUNE_NAMES); unnamed ones keep 0 (default)."""
        arr = np.array([int(values.get(k, 0)) for k in TUNE_NAMES], dtype=np.int32)
        _check(lib().stiv_set_tuning(self.h, arr.ctypes.data), "stiv_set_tuning")

    def result(self, counts, grad: bool) -> dict:
        b = self.buf
        npairs = int(counts[C_PAIRS])
        nc = int(counts[C_VF] + counts[C_EE])
        r = dict(counts=counts, i=b.ci[:npairs], j=b.cj[:npairs], shift=b.cs[:npairs], pair=b.pair[:nc],
                 type=b.type[:nc], a=b.a[:nc], b=b.b[:nc], tau=b.tau[:nc], w=b.w[:nc], V=b.Vc[:nc],
                 V_pair=b.Vp[:npairs])
        if grad:
            r.update(grad=b.grad[:nc], gves=b.gves[:nc], gvid=b.gvid[:nc])
        return r


def shift_vec(code):
    """shift code 9(sx+1) + 3(sy+1) + (sz+1) -> (sx, sy, sz) (numpy, vectorised)."""
    code = np.asarray(code)
    return np.stack([code // 9 - 1, (code // 3) % 3 - 1, code % 3 - 1], axis=-1)


class ContactLCP:
    """The contact LCP of a step (Eq. 3.7): 0 <= -V + B lambda perp lambda >= 0,
    B = J M J^T with M_ii = m_i I + t_i (1 1^T (x) I_3) per vesicle (m_i = 1
    when m_ves is None, t_i = 0 when t_ves is None).  Buffers grow when the
    library reports a capacity overflow."""

    def __init__(self, device="cuda", row_cap: int = 1024, nnz_cap: int = 1 << 15):
        self.device = torch.device(device)
        self._alloc(row_cap, nnz_cap)

    def _alloc(self, row_cap, nnz_cap):
        d = self.device
        self.row_cap, self.nnz_cap = int(row_cap), int(nnz_cap)
        self.row_pair = torch.zeros(self.row_cap, dtype=torch.int32, device=d)
        self.q = torch.zeros(self.row_cap, dtype=torch.float64, device=d)
        self.row_ptr = torch.zeros(self.row_cap + 1, dtype=torch.int64, device=d)
        self.col = torch.zeros(self.nnz_cap, dtype=torch.int32, device=d)
        self.val = torch.zeros(self.nnz_cap, dtype=torch.float64, device=d)
        self.dims = torch.zeros(8, dtype=torch.int64, device=d)
        self.lam = torch.zeros(self.row_cap, dtype=torch.float64, device=d)
        self.info = torch.zeros(4, dtype=torch.float64, device=d)

    def struct(self) -> StivLcp:
        return StivLcp(self.row_cap, self.nnz_cap, _ptr(self.row_pair), _ptr(self.q), _ptr(self.row_ptr),
                       _ptr(self.col), _ptr(self.val), _ptr(self.dims))

    def assemble(self, eng: "Stiv", ds: "DeviceScene", m_ves=None, t_ves=None, stream=None,
                 max_retries: int = 6) -> dict:
        """B and q from the engine's last step with grad=True (m_ves, t_ves:
        float64 device tensors [n] or None)."""
        b = eng.buf
        st = _stream(stream)
        mv = 0 if m_ves is None else _ptr(m_ves)
        tv = 0 if t_ves is None else _ptr(t_ves)
        for _ in range(max_retries):
            lcp = self.struct()
            _check(lib().stiv_lcp_matrix(eng.h, st, ds.n, ds.p_max, ctypes.byref(b.pairs_struct()),
                                         ctypes.byref(b.contacts_struct()), _ptr(b.counts), _ptr(b.Vp),
                                         _ptr(b.grad), _ptr(b.gves), _ptr(b.gvid), mv, tv, ctypes.byref(lcp)),
                   "stiv_lcp_matrix")
            dims = self.dims.cpu().numpy()
            if dims[2] == 0:
                n, nnz = int(dims[0]), int(dims[1])
                return dict(n=n, nnz=nnz, row_pair=self.row_pair[:n], q=self.q[:n], row_ptr=self.row_ptr[:n + 1],
                            col=self.col[:nnz], val=self.val[:nnz])
            self._alloc(max(self.row_cap, 2 * int(dims[0]) + 16) if dims[2] & 1 else self.row_cap,
                        max(self.nnz_cap, 2 * int(dims[1]) + 16) if dims[2] & 2 else self.nnz_cap)
        raise StivError(STIV_ERR_CAPACITY, "lcp: capacities kept overflowing")

    def load_csr(self, row_ptr, col, val, q):
        """A given matrix (CSR, host arrays) and q, for stiv_lcp_solve."""
        n, nnz = len(q), len(val)
        if n > self.row_cap or nnz > self.nnz_cap:
            self._alloc(max(self.row_cap, n), max(self.nnz_cap, nnz))
        d = self.device
        self.row_ptr[:n + 1].copy_(torch.as_tensor(np.asarray(row_ptr, dtype=np.int64), device=d))
        self.col[:nnz].copy_(torch.as_tensor(np.asarray(col, dtype=np.int32), device=d))
        self.val[:nnz].copy_(torch.as_tensor(np.asarray(val, dtype=np.float64), device=d))
        self.q[:n].copy_(torch.as_tensor(np.asarray(q, dtype=np.float64), device=d))
        self.dims.copy_(torch.tensor([n, nnz, 0, 0, 0, 0, 0, 0], dtype=torch.int64, device=d))

    def solve(self, eng: "Stiv", tol: float = 1e-12, max_newton: int = 100, max_cg: int = 2000,
              stream=None) -> dict:
        _check(lib().stiv_lcp_solve(eng.h, _stream(stream), ctypes.byref(self.struct()), float(tol), int(max_newton),
                                    int(max_cg), _ptr(self.lam), _ptr(self.info)), "stiv_lcp_solve")
        n = int(self.dims[0].item())
        info = self.info.cpu().numpy()
        return dict(lam=self.lam[:n], newton=int(info[0]), residual=float(info[1]), cg=int(info[2]),
                    status=int(info[3]))
