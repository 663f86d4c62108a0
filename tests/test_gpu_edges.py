"""Edge cases of the collision step through the C ABI, against the oracle:
no projectiles at all, single pairs, a lone projectile among many ions and
the reverse, the largest cell the binning supports (16384), the
small/large permutation boundary (32 / 33), and positrons present from the
start.  FP64 plain path bit-exact; FP32 batched path within its decision
bound."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1907_02814_gb300 import workloads as W  # noqa: E402


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


SHAPES = {"single": ([1], [1]), "lone_projectile": ([1], [1000]), "lone_ion": ([1000], [1]),
          "largest": ([16384], [3]), "perm_boundary": ([32, 33, 33, 32], [33, 32, 1, 1]),
          "mixed": ([0, 5, 0, 7, 64, 1], [3, 0, 0, 9, 2, 64])}


def workload(e, i, seed, positrons=False):
    e, i = np.array(e), np.array(i)
    wl = W.solid_cu(n_cells=len(e), e_per_cell=e, i_per_cell=i, seed=seed, dt=200e-15, T_mev=30.0,
                    photons_per_cell=np.maximum(e // 2, 1) * (i > 0))
    if positrons:
        em = wl.species["em"]
        k = len(em["w"]) // 3
        wl.species["ep"] = {f: (v[:k].copy() if v is not None else None) for f, v in em.items()}
        wl.species["ep"]["pid"] = wl.species["ep"]["pid"] + np.uint64(1 << 40)
    return wl


def run(pcc, ctx, orc, wl, precision):
    ctx.tables_build([pcc.material(m.Z, m.Zstar, m.n_i, m.T_e) for m in wl.materials],
                     pcc.table_spec(n_rows=64, n_cols=64))
    dev = {}
    for name, d in wl.species.items():
        n = len(d["w"])
        sp = pcc.DeviceSpecies.empty(wl.n_cells, n + 600 * wl.n_cells + n)
        if n:
            pcc.bin(ctx, pcc.particles_to_device(d), wl.n_cells, sp, slack_abs=600, slack_rel=1.0)
        else:
            pcc.bin(ctx, {"n": 0, "ux": None, "uy": None, "uz": None, "w": None, "pid": None, "cell": None},
                    wl.n_cells, sp, slack_abs=600, slack_rel=1.0)
        dev[name] = sp
    mat = torch.as_tensor(wl.material_of_cell, device="cuda")
    ctx.read_status()
    pcc.collide(ctx, wl.n_cells, mat, wl.ion_mass, dev["em"], dev["ep"], dev["ph"], dev["ion"], wl.dt, wl.seed, 0,
                precision=precision)
    for k in ("em", "ep", "ph"):
        pcc.append_secondaries(ctx, wl.n_cells, dev[k])
    status, stats = ctx.read_status()
    T = orc.OracleTables([orc.material(m.Z, m.Zstar, m.n_i, m.T_e) for m in wl.materials],
                         orc.table_spec(n_rows=64, n_cols=64))
    sp = {k: orc.OracleSpecies(v, cap=len(v["w"]) + 100000) for k, v in wl.species.items()}
    _, st = orc.step(T, wl.n_cells, wl.material_of_cell, sp["em"], sp["ep"], sp["ph"], sp["ion"], wl.ion_mass,
                     wl.dt, wl.seed, 0)
    return dev, status, stats, sp, st


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_edge_shapes(pcc, ctx, orc, shape, precision):
    e, i = SHAPES[shape]
    wl = workload(e, i, seed=10 + list(SHAPES).index(shape), positrons=(shape == "mixed"))
    prec = pcc.FP64_PLAIN if precision == "fp64" else pcc.FP32_BATCHED
    dev, status, stats, sp, st = run(pcc, ctx, orc, wl, prec)
    assert status & pcc.ST_CAPACITY == 0 and status & pcc.ST_NONFINITE == 0
    assert stats["pairs"] == [int(v) for v in st["pairs"]]
    pairs = sum(st["pairs"])
    if precision == "fp64":
        assert stats["created"] == [int(v) for v in st["created"]]
        for k in ("em", "ep", "ph"):
            g, o = dev[k].live_host(), sp[k].canonical()
            assert np.array_equal(g["pid"], o["pid"]), k
            for f in ("ux", "uy", "uz"):
                np.testing.assert_allclose(g[f], o[f], rtol=2e-6, atol=1e-6, err_msg=f"{k}.{f}")
    else:
        mism = sum(len(set(dev[k].live_host()["pid"].tolist()) ^ set(sp[k].canonical()["pid"].tolist()))
                   for k in ("em", "ep", "ph"))
        assert mism <= max(2, 1e-5 * pairs), (mism, pairs)


def test_no_projectiles(pcc, ctx, orc):
    """Cells with ions and no electrons, positrons or photons: nothing is
    paired, nothing changes, no status bit."""
    wl = W.solid_cu(n_cells=8, e_per_cell=0, i_per_cell=5, seed=3)
    for prec in (pcc.FP64_PLAIN, pcc.FP32_BATCHED):
        dev, status, stats, sp, st = run(pcc, ctx, orc, wl, prec)
        assert status == 0 and sum(stats["pairs"]) == 0 and sum(stats["created"]) == 0
        assert all(int(dev[k].cell_count.sum()) == 0 for k in ("em", "ep", "ph"))
