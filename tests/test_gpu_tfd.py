"""The TFD-quadrature screening mode on the GPU: tables whose relativistic
Brems and Bethe-Heitler rows use I1, I2 (Eqs. defphi1, defphi2) of the full
Thomas-Fermi-Debye potential, integrated by the table kernel, against the
oracle's own quadrature; the build time of both modes; and one collision
step on such tables against the oracle (FP64 plain path bit-exact, FP32
batched path within its decision bound)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1907_02814_gb300 import workloads as W  # noqa: E402

MATS = [W.Material(29, 5.0, 8.5e28, 100.0), W.Material(79, 30.0, 5.9e28, 1e3), W.Material(13, 0.0, 6e28, 1.0),
        W.Material(73, 73.0, 5.5e28, 1e4), W.Material(29, 14.5, 8.5e28, 5e3, 1.3, 0.7)]


@pytest.fixture(scope="module")
def pcc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_02814_gb300 import build, pcc as p
    build.build()
    return p


@pytest.fixture(scope="module")
def ctx(pcc):
    c = pcc.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("kw", [dict(n_rows=96, n_cols=80), dict(n_rows=256, n_cols=256)])
def test_tfd_tables_match_oracle(pcc, ctx, orc, kw):
    """Two independent quadratures of the same integrals (the kernel's unit
    panels in ln u with 12 nodes, the oracle's half-unit panels with 8):
    agreement to 1e-9, tighter than the reduced mode's 1e-7 because neither
    side evaluates the cancelling closed form of Eq. (deriv_I2)."""
    ctx.tables_build([pcc.material(m.Z, m.Zstar, m.n_i, m.T_e, m.s_TF, m.s_D) for m in MATS],
                     pcc.table_spec(screening=pcc.SCREEN_TFD_QUAD, **kw))
    g = ctx.tables_read()
    o = orc.OracleTables([orc.material(m.Z, m.Zstar, m.n_i, m.T_e, m.s_TF, m.s_D) for m in MATS],
                         orc.table_spec(screening=orc.SCREEN_TFD_QUAD, **kw))
    np.testing.assert_allclose(g["brems_sigma"], o.brems_sigma, rtol=1e-9)
    np.testing.assert_allclose(g["bh_sigma"], o.bh_sigma, rtol=1e-9)
    for k in ("brems_cdf", "bh_cdf", "tri_gp_cdf", "tri_split_cdf"):
        np.testing.assert_allclose(g[k], getattr(o, k), rtol=1e-9, atol=1e-12, err_msg=k)
    # the mode changes the tables where the potential has two terms
    ctx.tables_build([pcc.material(m.Z, m.Zstar, m.n_i, m.T_e, m.s_TF, m.s_D) for m in MATS], pcc.table_spec(**kw))
    r = ctx.tables_read()
    d = np.abs(r["bh_sigma"] / g["bh_sigma"] - 1.0).max(axis=1)
    assert d[0] > 1e-3 and d[2] < 1e-9      # Z* = 5 of 29 differs; Z* = 0 coincides


def test_table_build_time(pcc, ctx):
    mats = [pcc.material(29, 14.0, 8.5e28, 5e3)]
    out = {}
    for name, mode in (("reduced", pcc.SCREEN_REDUCED), ("tfd_quad", pcc.SCREEN_TFD_QUAD)):
        ctx.tables_build(mats, pcc.table_spec(screening=mode))
        torch.cuda.synchronize()
        t = time.perf_counter()
        ctx.tables_build(mats, pcc.table_spec(screening=mode))
        torch.cuda.synchronize()
        out[name] = (time.perf_counter() - t) * 1e3
    print(f"\n[TFD] 256 x 256 tables, one material: reduced {out['reduced']:.1f} ms, "
          f"TFD quadrature {out['tfd_quad']:.1f} ms")
    assert out["tfd_quad"] < 5000.0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_collide_on_tfd_tables(pcc, ctx, orc, precision):
    rng = np.random.default_rng(31)
    n = 48
    e = rng.integers(0, 300, n)
    wl = W.solid_cu(n_cells=n, e_per_cell=e, i_per_cell=rng.integers(1, 60, n), seed=31, dt=300e-15, T_mev=30.0,
                    Zstar=14.0, T_e=5e3, photons_per_cell=np.maximum(e // 2, 1))
    spec = dict(n_rows=96, n_cols=96)
    ctx.tables_build([pcc.material(m.Z, m.Zstar, m.n_i, m.T_e) for m in wl.materials],
                     pcc.table_spec(screening=pcc.SCREEN_TFD_QUAD, **spec))
    dev = {}
    for name, d in wl.species.items():
        cnt = len(d["w"])
        sp = pcc.DeviceSpecies.empty(wl.n_cells, cnt + 600 * wl.n_cells + cnt)
        if cnt:
            pcc.bin(ctx, pcc.particles_to_device(d), wl.n_cells, sp, slack_abs=600, slack_rel=1.0)
        else:
            pcc.bin(ctx, {"n": 0, "ux": None, "uy": None, "uz": None, "w": None, "pid": None, "cell": None},
                    wl.n_cells, sp, slack_abs=600, slack_rel=1.0)
        dev[name] = sp
    mat = torch.as_tensor(wl.material_of_cell, device="cuda")
    prec = pcc.FP64_PLAIN if precision == "fp64" else pcc.FP32_BATCHED
    ctx.read_status()
    pcc.collide(ctx, wl.n_cells, mat, wl.ion_mass, dev["em"], dev["ep"], dev["ph"], dev["ion"], wl.dt, wl.seed, 0,
                precision=prec)
    for k in ("em", "ep", "ph"):
        pcc.append_secondaries(ctx, wl.n_cells, dev[k])
    status, stats = ctx.read_status()
    T = orc.OracleTables([orc.material(m.Z, m.Zstar, m.n_i, m.T_e) for m in wl.materials],
                         orc.table_spec(screening=orc.SCREEN_TFD_QUAD, **spec))
    sp = {k: orc.OracleSpecies(v, cap=len(v["w"]) + 100000) for k, v in wl.species.items()}
    _, st = orc.step(T, wl.n_cells, wl.material_of_cell, sp["em"], sp["ep"], sp["ph"], sp["ion"], wl.ion_mass,
                     wl.dt, wl.seed, 0)
    assert status & (pcc.ST_CAPACITY | pcc.ST_NONFINITE) == 0, status
    assert stats["pairs"] == [int(v) for v in st["pairs"]]
    assert sum(int(v) for v in st["created"]) > 50
    if precision == "fp64":
        assert stats["created"] == [int(v) for v in st["created"]]
        for k in ("em", "ep", "ph"):
            g, o = dev[k].live_host(), sp[k].canonical()
            assert np.array_equal(g["pid"], o["pid"]), k
            for f in ("ux", "uy", "uz"):
                np.testing.assert_allclose(g[f], o[f], rtol=2e-6, atol=1e-6, err_msg=f"{k}.{f}")
    else:
        pairs = sum(int(v) for v in st["pairs"])
        mism = sum(len(set(dev[k].live_host()["pid"].tolist()) ^ set(sp[k].canonical()["pid"].tolist()))
                   for k in ("em", "ep", "ph"))
        assert mism <= max(2, 1e-5 * pairs), (mism, pairs)
