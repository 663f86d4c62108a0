"""ctypes front end of the FP64 CPU oracle (pcc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product library never imports
it.  The oracle shares no code with the CUDA path; see pcc_oracle.h.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, so x86 and Arm agree),
    with OpenMP over cells for timing when the compiler has it."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pcc_oracle.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Material(C.Structure):
    _fields_ = [("Z", C.c_int), ("Zstar", C.c_double), ("n_i", C.c_double), ("T_e", C.c_double),
                ("s_TF", C.c_double), ("s_D", C.c_double)]


class Screening(C.Structure):
    _fields_ = [("Z", C.c_int), ("Zstar", C.c_double), ("LTF", C.c_double), ("LD", C.c_double),
                ("etaTF", C.c_double), ("etaD", C.c_double), ("ITFD", C.c_double), ("LR", C.c_double),
                ("fC", C.c_double), ("lambdaD", C.c_double), ("ri", C.c_double), ("tfd_quad", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TableSpec(C.Structure):
    _fields_ = [("n_rows", C.c_int), ("n_cols", C.c_int), ("quad_nodes", C.c_int),
                ("T_min", C.c_double), ("T_max", C.c_double), ("x_min", C.c_double),
                ("tri_y_min", C.c_double), ("nr_qbounds", C.c_int), ("screening", C.c_int)]


_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)


class Tables(C.Structure):
    _fields_ = [("spec", TableSpec), ("n_mat", C.c_int), ("scr", C.POINTER(Screening)),
                ("brems_sigma", _dp), ("brems_cdf", _dp), ("bh_sigma", _dp), ("bh_cdf", _dp),
                ("tri_gp_cdf", _dp), ("tri_split_cdf", _dp)]


class Species(C.Structure):
    _fields_ = [("n", C.c_int), ("cap", C.c_int), ("ux", _fp), ("uy", _fp), ("uz", _fp), ("w", _fp),
                ("x", _fp), ("pid", C.POINTER(C.c_uint64)), ("cell", C.POINTER(C.c_int32))]


class Stats(C.Structure):
    _fields_ = [("pairs", C.c_double * 3), ("accepted", C.c_double * 5), ("created", C.c_double * 5),
                ("status", C.c_uint)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            d = C.c_double
            L.orc_screening_prep.argtypes = [C.POINTER(Material), C.POINTER(Screening)]
            L.orc_lambert_w0.restype = d; L.orc_lambert_w0.argtypes = [d]
            L.orc_fC.restype = d; L.orc_fC.argtypes = [C.c_int]
            for name in ("orc_I1_yukawa", "orc_I2_yukawa"):
                getattr(L, name).restype = d; getattr(L, name).argtypes = [d, d]
            L.orc_I_tfd.restype = d; L.orc_I_tfd.argtypes = [d, d, d, d]
            L.orc_I12_tfd_quad.argtypes = [C.POINTER(Screening), d, _dp, _dp]
            L.orc_dsdk_brems.restype = d; L.orc_dsdk_brems.argtypes = [C.POINTER(Screening), d, d, C.c_int]
            L.orc_dsdk_brems_nr.restype = d; L.orc_dsdk_brems_nr.argtypes = [C.POINTER(Screening), d, d, C.c_int]
            L.orc_dsdk_brems_rel.restype = d; L.orc_dsdk_brems_rel.argtypes = [C.POINTER(Screening), d, d, d]
            L.orc_dsdg_bh.restype = d; L.orc_dsdg_bh.argtypes = [C.POINTER(Screening), d, d]
            L.orc_sigma_trident.restype = d; L.orc_sigma_trident.argtypes = [C.c_int, d]
            L.orc_dsdgp_trident.restype = d; L.orc_dsdgp_trident.argtypes = [C.c_int, d, d]
            L.orc_split_shape.restype = d; L.orc_split_shape.argtypes = [d, d]
            L.orc_gauss_legendre.argtypes = [C.c_int, _dp, _dp]
            L.orc_row_value.restype = d; L.orc_row_value.argtypes = [C.POINTER(TableSpec), C.c_int]
            L.orc_col_value.restype = d; L.orc_col_value.argtypes = [C.POINTER(TableSpec), C.c_int, C.c_int]
            L.orc_tables_build.restype = C.c_int; L.orc_tables_build.argtypes = [C.POINTER(Tables)]
            u32p = C.POINTER(C.c_uint32)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_u01.restype = d; L.orc_u01.argtypes = [C.c_uint32]
            L.orc_accept.restype = C.c_int
            L.orc_accept.argtypes = [C.c_uint32, d, C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint64]
            L.orc_perm_pos.restype = C.c_uint32; L.orc_perm_pos.argtypes = [C.c_uint32, C.c_uint32, u32p]
            L.orc_perm_elem.restype = C.c_uint32; L.orc_perm_elem.argtypes = [C.c_uint32, C.c_uint32, u32p]
            L.orc_sigma_lookup.restype = d
            L.orc_sigma_lookup.argtypes = [C.POINTER(TableSpec), _dp, d, C.POINTER(C.c_uint)]
            L.orc_sample.restype = d
            L.orc_sample.argtypes = [C.POINTER(TableSpec), C.c_int, _dp, d, d, d]
            L.orc_step.restype = C.c_int
            L.orc_step.argtypes = [C.POINTER(Tables), C.c_int, C.POINTER(C.c_int32),
                                   C.POINTER(Species), C.POINTER(Species), C.POINTER(Species),
                                   C.POINTER(Species), d, d, C.c_uint64, C.c_uint64, C.c_uint, _dp,
                                   C.POINTER(Stats)]
            L.orc_boost.argtypes = [_dp, _dp, _dp, C.c_int]
            L.orc_expected_emission.argtypes = [C.POINTER(Material), C.c_int, _dp, _dp, C.c_int, _dp]
            L.orc_expected_emission_grad.argtypes = [C.POINTER(Material), C.c_int, _dp, _dp, C.c_int, _dp, _dp]
            L.orc_expected_emission_grad_analytic.argtypes = [C.POINTER(Material), C.c_int, _dp, _dp, C.c_int,
                                                              _dp, _dp]
            L.orc_dI12_dL.argtypes = [d, d, _dp, _dp]
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_get_threads.restype = C.c_int
            L.orc_dsdk_brems_grad.argtypes = [C.POINTER(Material), d, d, _dp]
            L.orc_screening_jacobian.argtypes = [C.POINTER(Material), _dp]
    return _lib


# ---------------------------------------------------------------- physics --
TB_BREMS, TB_BH, TB_TRI_GP, TB_TRI_SPLIT = 0, 1, 2, 3
NR_EXACT, NR_PRINTED = 0, 1
SCREEN_REDUCED, SCREEN_TFD_QUAD = 0, 1
PROC_BREMS, PROC_TRIDENT, PROC_BH = 1, 2, 4


def material(Z, Zstar, n_i, T_e, s_TF=1.0, s_D=1.0) -> Material:
    return Material(int(Z), float(Zstar), float(n_i), float(T_e), float(s_TF), float(s_D))


def screening(mat: Material) -> Screening:
    s = Screening()
    lib().orc_screening_prep(C.byref(mat), C.byref(s))
    return s


def lambert_w0(z):
    return lib().orc_lambert_w0(float(z))


def fC(Z):
    return lib().orc_fC(int(Z))


def I1(delta, L):
    return lib().orc_I1_yukawa(float(delta), float(L))


def I2(delta, L):
    return lib().orc_I2_yukawa(float(delta), float(L))


def I_tfd(etaTF, LTF, etaD, LD):
    return lib().orc_I_tfd(float(etaTF), float(LTF), float(etaD), float(LD))


def I12_tfd_quad(scr, delta):
    """(I1, I2) of Eqs. (defphi1), (defphi2) for the full TFD potential."""
    a, b = C.c_double(), C.c_double()
    lib().orc_I12_tfd_quad(C.byref(scr), float(delta), C.byref(a), C.byref(b))
    return a.value, b.value


def screening_tfd(mat: Material) -> Screening:
    """Screening of a material whose relativistic Brems and BH cross sections
    use the full TFD potential (I1, I2 by quadrature) instead of L_R."""
    s = screening(mat)
    s.tfd_quad = 1
    return s


def dsdk_brems(scr, gamma1, k, qb=NR_EXACT):
    return lib().orc_dsdk_brems(C.byref(scr), float(gamma1), float(k), int(qb))


def dsdk_brems_nr(scr, gamma1, k, qb=NR_EXACT):
    return lib().orc_dsdk_brems_nr(C.byref(scr), float(gamma1), float(k), int(qb))


def dsdk_brems_rel(scr, gamma1, k, fc=0.0):
    return lib().orc_dsdk_brems_rel(C.byref(scr), float(gamma1), float(k), float(fc))


def dsdg_bh(scr, k, gplus):
    return lib().orc_dsdg_bh(C.byref(scr), float(k), float(gplus))


def sigma_trident(Z, gamma1):
    return lib().orc_sigma_trident(int(Z), float(gamma1))


def dsdgp_trident(Z, gamma1, gp):
    return lib().orc_dsdgp_trident(int(Z), float(gamma1), float(gp))


def split_shape(gp, gplus):
    return lib().orc_split_shape(float(gp), float(gplus))


def gauss_legendre(n):
    x = np.zeros(n); w = np.zeros(n)
    lib().orc_gauss_legendre(n, x.ctypes.data_as(_dp), w.ctypes.data_as(_dp))
    return x, w


# ----------------------------------------------------------------- tables --
def table_spec(n_rows=256, n_cols=256, quad_nodes=8, gamma_min=1.002, gamma_max=2000.0,
               cutoff_exp=7, tri_y_min=1e-5, nr_qbounds=NR_EXACT, screening=SCREEN_REDUCED) -> TableSpec:
    return TableSpec(n_rows, n_cols, quad_nodes, gamma_min - 1.0, gamma_max - 1.0,
                     10.0 ** (-cutoff_exp), tri_y_min, nr_qbounds, screening)


class OracleTables:
    """Tables for a list of materials, built by the oracle in FP64."""

    def __init__(self, materials, spec: TableSpec):
        self.materials = list(materials)
        self.spec = spec
        n, R, Cn = len(self.materials), spec.n_rows, spec.n_cols
        self.scr_arr = (Screening * n)()
        for i, m in enumerate(self.materials):
            lib().orc_screening_prep(C.byref(m), C.byref(self.scr_arr[i]))
        self.brems_sigma = np.zeros((n, R)); self.brems_cdf = np.zeros((n, R, Cn))
        self.bh_sigma = np.zeros((n, R)); self.bh_cdf = np.zeros((n, R, Cn))
        self.tri_gp_cdf = np.zeros((R, Cn)); self.tri_split_cdf = np.zeros((R, Cn))
        self.c = Tables(spec, n, self.scr_arr,
                        self.brems_sigma.ctypes.data_as(_dp), self.brems_cdf.ctypes.data_as(_dp),
                        self.bh_sigma.ctypes.data_as(_dp), self.bh_cdf.ctypes.data_as(_dp),
                        self.tri_gp_cdf.ctypes.data_as(_dp), self.tri_split_cdf.ctypes.data_as(_dp))
        rc = lib().orc_tables_build(C.byref(self.c))
        if rc != 0:
            raise ValueError("oracle table build rejected the spec")

    def screening(self, i):
        return self.scr_arr[i]

    def row_value(self, r):
        return lib().orc_row_value(C.byref(self.spec), int(r))

    def col_value(self, table, c):
        return lib().orc_col_value(C.byref(self.spec), int(table), int(c))

    def sigma_lookup(self, which, mat, r):
        st = C.c_uint(0)
        arr = self.brems_sigma if which == TB_BREMS else self.bh_sigma
        row = np.ascontiguousarray(arr[mat])
        v = lib().orc_sigma_lookup(C.byref(self.spec), row.ctypes.data_as(_dp), float(r), C.byref(st))
        return v, st.value

    def sample(self, table, mat, r, u_row, u_col):
        if table == TB_BREMS:
            arr = self.brems_cdf[mat]
        elif table == TB_BH:
            arr = self.bh_cdf[mat]
        elif table == TB_TRI_GP:
            arr = self.tri_gp_cdf
        else:
            arr = self.tri_split_cdf
        arr = np.ascontiguousarray(arr)
        return lib().orc_sample(C.byref(self.spec), int(table), arr.ctypes.data_as(_dp), float(r),
                                float(u_row), float(u_col))


# ------------------------------------------------------------------- RNG --
def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [o[i] for i in range(4)]


def u01(r):
    return lib().orc_u01(int(r) & 0xFFFFFFFF)


def accept(a, p, c0, cell, step, tag, seed):
    """The accept decision U < p with U = (2^48 a + e + 1/2) 2^-64: a the
    16-bit first digit, e = 2^16 w0 + (w1 >> 16) from words w0, w1 of the draw
    (c0, cell, step, tag) under the key seed."""
    if not 0 <= int(a) < 1 << 16:
        raise ValueError("the first digit has 16 bits")
    return bool(lib().orc_accept(int(a), float(p), int(c0), int(cell), int(step), int(tag), int(seed)))


def perm_pos(s, n, rk):
    a = (C.c_uint32 * 4)(*rk)
    return lib().orc_perm_pos(int(s), int(n), a)


def perm_elem(j, n, rk):
    a = (C.c_uint32 * 4)(*rk)
    return lib().orc_perm_elem(int(j), int(n), a)


# ------------------------------------------------------------------ step --
SPECIES_FIELDS = ("ux", "uy", "uz", "w", "x", "pid", "cell")


class OracleSpecies:
    """Host copy of one particle population with spare capacity for appends."""

    def __init__(self, d: dict, cap: int | None = None):
        n = len(d["w"])
        cap = max(n, cap if cap is not None else n)
        self.n = n
        self.cap = cap
        self.ux = np.zeros(cap, np.float32); self.ux[:n] = d["ux"]
        self.uy = np.zeros(cap, np.float32); self.uy[:n] = d["uy"]
        self.uz = np.zeros(cap, np.float32); self.uz[:n] = d["uz"]
        self.w = np.zeros(cap, np.float32); self.w[:n] = d["w"]
        self.has_x = d.get("x") is not None
        self.x = np.zeros(cap, np.float32)
        if self.has_x:
            self.x[:n] = d["x"]
        self.pid = np.zeros(cap, np.uint64); self.pid[:n] = d["pid"]
        self.cell = np.zeros(cap, np.int32); self.cell[:n] = d["cell"]

    def cstruct(self):
        return Species(self.n, self.cap, self.ux.ctypes.data_as(_fp), self.uy.ctypes.data_as(_fp),
                       self.uz.ctypes.data_as(_fp), self.w.ctypes.data_as(_fp),
                       self.x.ctypes.data_as(_fp) if self.has_x else None,
                       self.pid.ctypes.data_as(C.POINTER(C.c_uint64)),
                       self.cell.ctypes.data_as(C.POINTER(C.c_int32)))

    def as_dict(self):
        n = self.n
        d = {k: getattr(self, k)[:n].copy() for k in ("ux", "uy", "uz", "w", "pid", "cell")}
        d["x"] = self.x[:n].copy() if self.has_x else None
        return d

    def canonical(self):
        """Arrays sorted by (cell, pid), the order the product stores them in."""
        d = self.as_dict()
        order = np.lexsort((d["pid"], d["cell"]))
        return {k: (v[order] if v is not None else None) for k, v in d.items()}


def set_threads(n: int) -> int:
    """Threads for the cells of a group in step() (timing only: the result
    does not depend on it); returns the count in effect (1 without OpenMP)."""
    lib().orc_set_threads(int(n))
    return int(lib().orc_get_threads())


def step(tables: OracleTables, n_cells, material_of_cell, em, ep, ph, ion, ion_mass, dt, seed,
         step_index, mask=PROC_BREMS | PROC_TRIDENT | PROC_BH, ledger=None):
    """One collision step; em/ep/ph are OracleSpecies updated in place."""
    mat = np.ascontiguousarray(material_of_cell, dtype=np.int32)
    if ledger is None:
        ledger = np.zeros((n_cells, 2))
    st = Stats()
    s_em, s_ep, s_ph, s_ion = em.cstruct(), ep.cstruct(), ph.cstruct(), ion.cstruct()
    rc = lib().orc_step(C.byref(tables.c), int(n_cells), mat.ctypes.data_as(C.POINTER(C.c_int32)),
                        C.byref(s_em), C.byref(s_ep), C.byref(s_ph), C.byref(s_ion), float(ion_mass),
                        float(dt), C.c_uint64(int(seed)), C.c_uint64(int(step_index)), int(mask),
                        ledger.ctypes.data_as(_dp), C.byref(st))
    em.n, ep.n, ph.n = s_em.n, s_ep.n, s_ph.n
    stats = {"pairs": list(st.pairs), "accepted": list(st.accepted), "created": list(st.created),
             "status": st.status, "rc": rc}
    return ledger, stats


def boost(ui, four, inverse=False):
    a = np.ascontiguousarray(ui, dtype=np.float64)
    b = np.ascontiguousarray(four, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_boost(a.ctypes.data_as(_dp), b.ctypes.data_as(_dp), out.ctypes.data_as(_dp), int(inverse))
    return out


def expected_emission(mat: Material, gamma, w, n_quad=64):
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_expected_emission(C.byref(mat), len(g), g.ctypes.data_as(_dp), ww.ctypes.data_as(_dp),
                                int(n_quad), out.ctypes.data_as(_dp))
    return out


def expected_emission_grad(mat: Material, gamma, w, g_out, n_quad=64):
    """sum_j g_out[j] d out[j] / d (n_i, T_e, Z*, s_TF, s_D), FP64."""
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    go = np.ascontiguousarray(g_out, dtype=np.float64)
    out = np.zeros(5)
    lib().orc_expected_emission_grad(C.byref(mat), len(g), g.ctypes.data_as(_dp), ww.ctypes.data_as(_dp),
                                     int(n_quad), go.ctypes.data_as(_dp), out.ctypes.data_as(_dp))
    return out



def expected_emission_grad_analytic(mat: Material, gamma, w, g_out, n_quad=64):
    """sum_j g_out[j] d out[j] / d (n_i, T_e, Z*, s_TF, s_D) by the chain rule
    written out by hand (FP64)."""
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    go = np.ascontiguousarray(g_out, dtype=np.float64)
    out = np.zeros(5)
    lib().orc_expected_emission_grad_analytic(C.byref(mat), len(g), g.ctypes.data_as(_dp), ww.ctypes.data_as(_dp),
                                              int(n_quad), go.ctypes.data_as(_dp), out.ctypes.data_as(_dp))
    return out


def dI12_dL(delta, L):
    a, b = C.c_double(), C.c_double()
    lib().orc_dI12_dL(float(delta), float(L), C.byref(a), C.byref(b))
    return a.value, b.value


def dsdk_brems_grad(mat: Material, gamma1, k):
    """d(dsigma/dk)/d(L_TF, L_D, eta_D, L_R)."""
    out = np.zeros(4)
    lib().orc_dsdk_brems_grad(C.byref(mat), float(gamma1), float(k), out.ctypes.data_as(_dp))
    return out


def screening_jacobian(mat: Material):
    """d(L_TF, L_D, eta_D, L_R)/d(n_i, T_e, Z*, s_TF, s_D) as a 4 x 5 array."""
    out = np.zeros(20)
    lib().orc_screening_jacobian(C.byref(mat), out.ctypes.data_as(_dp))
    return out.reshape(4, 5)
