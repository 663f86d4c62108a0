"""Thin ctypes binding of the C ABI in include/pcc.h.

Argument marshalling only: every step of the collision path runs in the
CUDA kernels of libpcc.so.  PyTorch tensors supply device memory and the
current CUDA stream.  There is no CPU fallback: importing the compute
functions without a built library raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpcc.so")

PCC_OK, PCC_E_INVALID, PCC_E_CUDA, PCC_E_CAPACITY, PCC_E_NO_TABLES = 0, 1, 2, 3, 4
ST_TABLE_RANGE, ST_PROB_LARGE, ST_CAPACITY, ST_NONFINITE, ST_ID_RANGE, ST_TIMEOUT = 1, 2, 4, 8, 16, 32
ST_BOUND_RANGE = 64
FP64_PLAIN, FP32_BATCHED = 0, 1
BREMS, TRIDENT, BH = 1, 2, 4
GROUP_EM, GROUP_EP, GROUP_PH = 0x100, 0x200, 0x400

_vp = C.c_void_p
_fp = C.POINTER(C.c_float)


class Material(C.Structure):
    _fields_ = [("Z", C.c_int), ("Zstar", C.c_double), ("n_i", C.c_double), ("T_e", C.c_double),
                ("s_TF", C.c_double), ("s_D", C.c_double)]


class TableSpec(C.Structure):
    _fields_ = [("n_rows", C.c_int), ("n_cols", C.c_int), ("quad_nodes", C.c_int), ("gamma_min", C.c_double),
                ("gamma_max", C.c_double), ("cutoff_exp", C.c_int), ("tri_y_min", C.c_double),
                ("nr_qbounds", C.c_int), ("screening", C.c_int)]


class Species(C.Structure):
    _fields_ = [("ux", _vp), ("uy", _vp), ("uz", _vp), ("w", _vp), ("x", _vp), ("pid", _vp),
                ("cell_start", _vp), ("cell_count", _vp), ("cell_added", _vp), ("capacity", C.c_int)]


class Particles(C.Structure):
    _fields_ = [("n", C.c_int), ("ux", _vp), ("uy", _vp), ("uz", _vp), ("w", _vp), ("x", _vp), ("pid", _vp),
                ("cell", _vp)]


class Cells(C.Structure):
    _fields_ = [("n_cells", C.c_int), ("material_of_cell", _vp), ("ion_mass", C.c_double)]


class StepDesc(C.Structure):
    _fields_ = [("cells", C.POINTER(Cells)), ("em", C.POINTER(Species)), ("ep", C.POINTER(Species)),
                ("ph", C.POINTER(Species)), ("ion", C.POINTER(Species)), ("dt", C.c_double), ("seed", C.c_uint64),
                ("mask", C.c_uint), ("precision", C.c_int), ("ledger", _vp)]


class Stats(C.Structure):
    _fields_ = [("pairs", C.c_ulonglong * 3), ("accepted", C.c_ulonglong * 5), ("created", C.c_ulonglong * 5),
                ("energy_change", C.c_double), ("charge_change", C.c_double), ("candidates", C.c_ulonglong * 3)]


_lib = None

EXPORTS = {
    "pcc_version": (C.c_char_p, []),
    "pcc_last_error": (C.c_char_p, []),
    "pcc_status_string": (C.c_char_p, [C.c_int]),
    "pcc_status_bit_string": (C.c_char_p, [C.c_uint]),
    "pcc_create": (C.c_int, [C.POINTER(_vp), C.c_int]),
    "pcc_destroy": (None, [_vp]),
    "pcc_tables_build": (C.c_int, [_vp, C.POINTER(Material), C.c_int, C.POINTER(TableSpec), _vp]),
    "pcc_tables_read": (C.c_int, [_vp] + [_vp] * 7),
    "pcc_bin": (C.c_int, [_vp, C.POINTER(Particles), C.c_int, C.POINTER(Species), C.c_int, C.c_double, _vp]),
    "pcc_collide": (C.c_int, [_vp, C.POINTER(Cells), C.POINTER(Species), C.POINTER(Species), C.POINTER(Species),
                              C.POINTER(Species), C.c_double, C.c_uint64, C.c_uint64, C.c_uint, C.c_int, _vp, _vp]),
    "pcc_append_secondaries": (C.c_int, [_vp, C.c_int, C.POINTER(Species), _vp]),
    "pcc_set_schedule": (C.c_int, [_vp, C.c_int, C.c_int]),
    "pcc_set_scan_classes": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int)]),
    "pcc_get_scan_classes": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int)]),
    "pcc_set_wait_limit": (C.c_int, [_vp, C.c_int]),
    "pcc_pairing": (C.c_int, [_vp, C.c_int, C.POINTER(Species), C.POINTER(Species), C.c_int, C.c_uint64,
                              C.c_uint64, _vp, _vp, _vp]),
    "pcc_totals": (C.c_int, [_vp, C.c_int, C.POINTER(Species), C.c_int, _vp, _vp]),
    "pcc_accept_check": (C.c_int, [C.c_int, _vp, _vp, _vp, _vp, _vp, C.c_uint64, C.c_uint64, _vp, _vp, _vp]),
    "pcc_totals_noalloc": (C.c_int, [C.c_int, C.POINTER(Species), C.c_int, _vp, _vp]),
    "pcc_read_status": (C.c_int, [_vp, C.POINTER(C.c_uint), C.POINTER(Stats), _vp]),
    "pcc_steps_capture": (C.c_int, [_vp, C.POINTER(StepDesc), C.c_uint64, C.c_int, C.c_int, _vp]),
    "pcc_steps_launch": (C.c_int, [_vp, _vp]),
    "pcc_steps_timing": (C.c_int, [_vp, _fp]),
    "pcc_launch_count": (C.c_ulonglong, []),
    "pcc_expected_emission_fwd": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp]),
    "pcc_expected_emission_bwd": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp,
                                            _vp]),
}


def load(path: str | None = None):
    """Load libpcc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run paper_1907_02814_gb300.build.build() first")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PccError(RuntimeError):
    pass


def status_string(code: int) -> str:
    """Name and meaning of a return code of the C ABI."""
    return load().pcc_status_string(int(code)).decode()


def status_bits(status: int) -> list[str]:
    """Names of the bits set in a device status word (pcc_read_status)."""
    L = load()
    return [L.pcc_status_bit_string(1 << b).decode() for b in range(32) if (int(status) >> b) & 1]


def _check(rc, what):
    if rc != PCC_OK:
        msg = load().pcc_last_error().decode()
        raise PccError(f"{what} failed with {status_string(rc)}: {msg}")


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def material(Z, Zstar, n_i, T_e, s_TF=1.0, s_D=1.0) -> Material:
    return Material(int(Z), float(Zstar), float(n_i), float(T_e), float(s_TF), float(s_D))


SCREEN_REDUCED, SCREEN_TFD_QUAD = 0, 1


def table_spec(n_rows=256, n_cols=256, quad_nodes=8, gamma_min=1.002, gamma_max=2000.0, cutoff_exp=7,
               tri_y_min=1e-5, nr_qbounds=0, screening=SCREEN_REDUCED) -> TableSpec:
    return TableSpec(n_rows, n_cols, quad_nodes, gamma_min, gamma_max, cutoff_exp, tri_y_min, nr_qbounds,
                     screening)


class Context:
    """A library context on one CUDA device (tables, status, scratch)."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = C.c_void_p()
        _check(self.lib.pcc_create(C.byref(h), int(device)), "pcc_create")
        self.h = h
        self.device = device
        self.spec = None
        self.n_mat = 0
        self.graph_steps = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.pcc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tables_build(self, materials, spec: TableSpec | None = None, stream=None):
        spec = spec or table_spec()
        arr = (Material * len(materials))(*materials)
        _check(self.lib.pcc_tables_build(self.h, arr, len(materials), C.byref(spec), _stream(stream)),
               "pcc_tables_build")
        self.spec = spec
        self.n_mat = len(materials)

    def tables_read(self):
        R, Cn, M = self.spec.n_rows, self.spec.n_cols, self.n_mat
        out = {"brems_sigma": np.zeros((M, R)), "brems_cdf": np.zeros((M, R, Cn)), "bh_sigma": np.zeros((M, R)),
               "bh_cdf": np.zeros((M, R, Cn)), "tri_gp_cdf": np.zeros((R, Cn)), "tri_split_cdf": np.zeros((R, Cn)),
               "screening": np.zeros((M, 8))}
        keys = ["brems_sigma", "brems_cdf", "bh_sigma", "bh_cdf", "tri_gp_cdf", "tri_split_cdf", "screening"]
        _check(self.lib.pcc_tables_read(self.h, *[C.c_void_p(out[k].ctypes.data) for k in keys]),
               "pcc_tables_read")
        return out

    def set_schedule(self, min_blocks_per_sm=4, blocks_per_sm=0):
        _check(self.lib.pcc_set_schedule(self.h, int(min_blocks_per_sm), int(blocks_per_sm)), "pcc_set_schedule")

    def set_scan_classes(self, group, thresholds):
        """Lane groups of the batched scan for group 0 (e-), 1 (e+) or 2
        (photons): size classes {warp, g16, g8, g4} (see pcc.h)."""
        arr = (C.c_int * 4)(*[int(v) for v in thresholds])
        _check(self.lib.pcc_set_scan_classes(self.h, int(group), arr), "pcc_set_scan_classes")

    def scan_classes(self, group):
        arr = (C.c_int * 4)()
        _check(self.lib.pcc_get_scan_classes(self.h, int(group), arr), "pcc_get_scan_classes")
        return [arr[i] for i in range(4)]

    def set_wait_limit(self, polls=1 << 22):
        """Fault injection: bounded waits give up after `polls` polls (0: at once)."""
        _check(self.lib.pcc_set_wait_limit(self.h, int(polls)), "pcc_set_wait_limit")

    def steps_capture(self, n_cells, material_of_cell, ion_mass, em, ep, ph, ion, dt, seed, step0, n_steps,
                      mask=BREMS | TRIDENT | BH, precision=FP32_BATCHED, ledger=None, timing=False, stream=None):
        """Capture n_steps full steps (collide of each group, then the three
        commits) into one CUDA graph held by the context."""
        cells = Cells(int(n_cells), _ptr(material_of_cell), float(ion_mass))
        sp = [x.cstruct() for x in (em, ep, ph, ion)]
        # the structs must outlive the call only; the graph keeps the device pointers
        d = StepDesc(C.pointer(cells), C.pointer(sp[0]), C.pointer(sp[1]), C.pointer(sp[2]), C.pointer(sp[3]),
                     float(dt), C.c_uint64(int(seed)), int(mask), int(precision), _ptr(ledger))
        _check(self.lib.pcc_steps_capture(self.h, C.byref(d), C.c_uint64(int(step0)), int(n_steps),
                                          int(bool(timing)), _stream(stream)), "pcc_steps_capture")
        self.graph_steps = int(n_steps)

    def steps_launch(self, stream=None):
        _check(self.lib.pcc_steps_launch(self.h, _stream(stream)), "pcc_steps_launch")

    def steps_timing(self):
        """[n_steps][4] milliseconds: e- group, e+ group, photon group, commits."""
        out = np.zeros((self.graph_steps, 4), dtype=np.float32)
        _check(self.lib.pcc_steps_timing(self.h, out.ctypes.data_as(_fp)), "pcc_steps_timing")
        return out

    def read_status(self, stream=None):
        st = C.c_uint(0)
        s = Stats()
        _check(self.lib.pcc_read_status(self.h, C.byref(st), C.byref(s), _stream(stream)), "pcc_read_status")
        return st.value, {"pairs": list(s.pairs), "accepted": list(s.accepted), "created": list(s.created),
                          "energy_change": s.energy_change, "charge_change": s.charge_change,
                          "candidates": list(s.candidates)}


@dataclass
class DeviceSpecies:
    """A species in cell-region layout held in torch tensors (device)."""
    ux: object
    uy: object
    uz: object
    w: object
    pid: object            # int64 tensor holding the uint64 bit patterns
    cell_start: object     # int32 [n_cells + 1]
    cell_count: object     # int32 [n_cells]
    cell_added: object     # int32 [n_cells]
    x: object = None

    @property
    def capacity(self):
        return int(self.w.numel())

    @staticmethod
    def empty(n_cells, capacity, device="cuda", with_x=False):
        import torch
        f = lambda: torch.zeros(capacity, dtype=torch.float32, device=device)
        return DeviceSpecies(f(), f(), f(), f(), torch.zeros(capacity, dtype=torch.int64, device=device),
                             torch.zeros(n_cells + 1, dtype=torch.int32, device=device),
                             torch.zeros(n_cells, dtype=torch.int32, device=device),
                             torch.zeros(n_cells, dtype=torch.int32, device=device),
                             f() if with_x else None)

    def cstruct(self) -> Species:
        return Species(_ptr(self.ux), _ptr(self.uy), _ptr(self.uz), _ptr(self.w), _ptr(self.x), _ptr(self.pid),
                       _ptr(self.cell_start), _ptr(self.cell_count), _ptr(self.cell_added), self.capacity)

    def live_host(self):
        """Live particles copied to the host in storage order (cell, pid)."""
        start = self.cell_start.cpu().numpy()
        count = self.cell_count.cpu().numpy()
        n_cells = len(count)
        idx = np.concatenate([np.arange(start[c], start[c] + count[c]) for c in range(n_cells)]) \
            if n_cells else np.zeros(0, np.int64)
        idx = idx.astype(np.int64)
        out = {k: getattr(self, k).cpu().numpy()[idx] for k in ("ux", "uy", "uz", "w")}
        out["pid"] = self.pid.cpu().numpy()[idx].view(np.uint64)
        out["cell"] = np.repeat(np.arange(n_cells, dtype=np.int32), count)
        out["x"] = self.x.cpu().numpy()[idx] if self.x is not None else None
        return out


def particles_to_device(d: dict, device="cuda"):
    """Host particle dict (workloads format) -> device tensors for pcc_bin."""
    import torch
    t = {k: torch.as_tensor(np.ascontiguousarray(d[k]), device=device) for k in ("ux", "uy", "uz", "w")}
    t["pid"] = torch.as_tensor(np.ascontiguousarray(d["pid"]).view(np.int64), device=device)
    t["cell"] = torch.as_tensor(np.ascontiguousarray(d["cell"], dtype=np.int32), device=device)
    t["x"] = torch.as_tensor(np.ascontiguousarray(d["x"]), device=device) if d.get("x") is not None else None
    t["n"] = len(d["w"])
    return t


def bin(ctx: Context, parts: dict, n_cells: int, out: DeviceSpecies, slack_abs=8, slack_rel=0.25, stream=None):
    p = Particles(int(parts["n"]), _ptr(parts["ux"]), _ptr(parts["uy"]), _ptr(parts["uz"]), _ptr(parts["w"]),
                  _ptr(parts.get("x")), _ptr(parts["pid"]), _ptr(parts["cell"]))
    s = out.cstruct()
    _check(ctx.lib.pcc_bin(ctx.h, C.byref(p), int(n_cells), C.byref(s), int(slack_abs), float(slack_rel),
                           _stream(stream)), "pcc_bin")


def collide(ctx: Context, n_cells: int, material_of_cell, ion_mass: float, em: DeviceSpecies, ep: DeviceSpecies,
            ph: DeviceSpecies, ion: DeviceSpecies, dt: float, seed: int, step: int, mask=BREMS | TRIDENT | BH,
            precision=FP32_BATCHED, ledger=None, stream=None):
    cells = Cells(int(n_cells), _ptr(material_of_cell), float(ion_mass))
    s = [x.cstruct() for x in (em, ep, ph, ion)]
    _check(ctx.lib.pcc_collide(ctx.h, C.byref(cells), C.byref(s[0]), C.byref(s[1]), C.byref(s[2]), C.byref(s[3]),
                               float(dt), C.c_uint64(int(seed)), C.c_uint64(int(step)), int(mask), int(precision),
                               _ptr(ledger), _stream(stream)), "pcc_collide")


def append_secondaries(ctx: Context, n_cells: int, sp: DeviceSpecies, stream=None):
    s = sp.cstruct()
    _check(ctx.lib.pcc_append_secondaries(ctx.h, int(n_cells), C.byref(s), _stream(stream)),
           "pcc_append_secondaries")


def pairing(ctx: Context, n_cells, proj: DeviceSpecies, targ: DeviceSpecies, group, seed, step, stream=None):
    import torch
    oj = torch.full((proj.capacity,), -1, dtype=torch.int32, device=proj.w.device)
    ot = torch.full((proj.capacity,), -1, dtype=torch.int32, device=proj.w.device)
    a, b = proj.cstruct(), targ.cstruct()
    _check(ctx.lib.pcc_pairing(ctx.h, int(n_cells), C.byref(a), C.byref(b), int(group), C.c_uint64(int(seed)),
                               C.c_uint64(int(step)), _ptr(oj), _ptr(ot), _stream(stream)), "pcc_pairing")
    return oj, ot


def accept_check(r, p, c0, cell, tag, step, seed, stream=None):
    """The kernels' accept decision U < p for device tensors r (int32, the
    16-bit accept digits), p (float64), c0, cell, tag (int32 views of the
    uint32 counter words); returns (out32, out64) int32 tensors of 0/1."""
    import torch
    n = int(r.numel())
    o32 = torch.zeros(n, dtype=torch.int32, device=r.device)
    o64 = torch.zeros(n, dtype=torch.int32, device=r.device)
    for t, dt in ((r, torch.int32), (p, torch.float64), (c0, torch.int32), (cell, torch.int32), (tag, torch.int32)):
        if t.dtype != dt or not t.is_contiguous() or t.numel() != n:
            raise PccError("accept_check: arrays must be contiguous, of equal length, int32 or float64 (p)")
    _check(load().pcc_accept_check(n, _ptr(r), _ptr(p), _ptr(c0), _ptr(cell), _ptr(tag),
                                   C.c_uint64(int(step)), C.c_uint64(int(seed)), _ptr(o32), _ptr(o64),
                                   _stream(stream)), "pcc_accept_check")
    return o32, o64


def totals(ctx: Context, n_cells, sp: DeviceSpecies, is_photon=False, stream=None):
    import torch
    out = torch.zeros(3, dtype=torch.float64, device=sp.w.device)
    s = sp.cstruct()
    _check(ctx.lib.pcc_totals(ctx.h, int(n_cells), C.byref(s), int(bool(is_photon)), _ptr(out), _stream(stream)),
           "pcc_totals")
    return out


def launch_count() -> int:
    """Kernels enqueued by the library so far in this process."""
    return int(load().pcc_launch_count())


def totals_noalloc(n_cells, sp: DeviceSpecies, out, is_photon=False, stream=None):
    """Allocation-free totals into the caller's device double[3] `out`."""
    s = sp.cstruct()
    _check(load().pcc_totals_noalloc(int(n_cells), C.byref(s), int(bool(is_photon)), _ptr(out), _stream(stream)),
           "pcc_totals_noalloc")
    return out


def _f32_cuda(name, t):
    import torch
    if t.dtype != torch.float32 or not t.is_cuda:
        raise TypeError(f"{name} must be a float32 CUDA tensor")
    return t.contiguous()


def expected_emission_fwd(ctx: Context, Z, params, gamma, w, n_quad=64, stream=None):
    import torch
    params, gamma, w = _f32_cuda("params", params), _f32_cuda("gamma", gamma), _f32_cuda("w", w)
    n_cells, n_samples = gamma.shape
    out = torch.empty((n_cells, 3), dtype=torch.float32, device=gamma.device)
    _check(ctx.lib.pcc_expected_emission_fwd(ctx.h, n_cells, n_samples, int(Z), int(n_quad), _ptr(params),
                                             _ptr(gamma), _ptr(w), _ptr(out), _stream(stream)),
           "pcc_expected_emission_fwd")
    return out


def expected_emission_bwd(ctx: Context, Z, params, gamma, w, grad_out, n_quad=64, stream=None):
    import torch
    params, gamma, w = _f32_cuda("params", params), _f32_cuda("gamma", gamma), _f32_cuda("w", w)
    grad_out = _f32_cuda("grad_out", grad_out)
    n_cells, n_samples = gamma.shape
    g = torch.empty((n_cells, 5), dtype=torch.float32, device=gamma.device)
    _check(ctx.lib.pcc_expected_emission_bwd(ctx.h, n_cells, n_samples, int(Z), int(n_quad), _ptr(params),
                                             _ptr(gamma), _ptr(w), _ptr(grad_out), _ptr(g),
                                             _stream(stream)), "pcc_expected_emission_bwd")
    return g
