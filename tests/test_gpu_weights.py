"""Unequal macro-particle weights through the C ABI, against the oracle.

With unequal target weights n_pt (Sec. III.A) is the sum of min(W_p, W_t)
over the actual pairs, so the pairing permutation enters the coefficient.
The cells span the size classes of every lane-group width of the batched
scan (whole warps, 16-, 8-, 4- and 2-lane groups), both pairing cases, the
rank-key and Feistel permutations (lists of at most 32 and of more), and
mix equal- and unequal-weight cells in the same warps.  FP64 plain path
bit-exact; FP32 batched path within its decision bound."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1907_02814_gb300 import workloads as W  # noqa: E402

FIXED = [(1, 1), (3, 7), (7, 2), (12, 30), (30, 12), (31, 31), (33, 5), (5, 33), (40, 60), (63, 63),
         (64, 2), (2, 64), (200, 40), (40, 200), (1, 90), (90, 1), (600, 40), (40, 600), (700, 3)]


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


def workload(seed=21, n_random=176):
    rng = np.random.default_rng(seed)
    e = np.concatenate([[p for p, _ in FIXED], rng.integers(0, 260, n_random)])
    i = np.concatenate([[t for _, t in FIXED], rng.integers(1, 90, n_random)])
    wl = W.solid_cu(n_cells=len(e), e_per_cell=e, i_per_cell=i, seed=seed, dt=200e-15, T_mev=30.0,
                    photons_per_cell=np.maximum(e // 2, 1) * (i > 0))
    # odd cells: target weights spread over a factor 4; every projectile
    # weight spread over a factor 2
    ion = wl.species["ion"]
    odd = (ion["cell"] % 2) == 1
    ion["w"] = np.where(odd, ion["w"] * rng.uniform(0.5, 2.0, len(ion["w"])), ion["w"]).astype(np.float32)
    for k in ("em", "ph"):
        d = wl.species[k]
        d["w"] = (d["w"] * rng.uniform(0.7, 1.4, len(d["w"]))).astype(np.float32)
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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_unequal_weights(pcc, ctx, orc, precision):
    wl = workload()
    prec = pcc.FP64_PLAIN if precision == "fp64" else pcc.FP32_BATCHED
    dev, status, stats, sp, st = run(pcc, ctx, orc, wl, prec)
    assert status & (pcc.ST_CAPACITY | pcc.ST_NONFINITE) == 0, status
    assert stats["pairs"] == [int(v) for v in st["pairs"]]
    assert sum(int(v) for v in st["created"]) > 50
    if precision == "fp64":
        assert stats["created"] == [int(v) for v in st["created"]]
        for k in ("em", "ep", "ph"):
            g, o = dev[k].live_host(), sp[k].canonical()
            assert np.array_equal(g["pid"], o["pid"]), k
            assert np.array_equal(g["w"], o["w"]), k
            for f in ("ux", "uy", "uz"):
                np.testing.assert_allclose(g[f], o[f], rtol=2e-6, atol=1e-6, err_msg=f"{k}.{f}")
    else:
        pairs = sum(int(v) for v in st["pairs"])
        mism = sum(len(set(dev[k].live_host()["pid"].tolist()) ^ set(sp[k].canonical()["pid"].tolist()))
                   for k in ("em", "ep", "ph"))
        assert mism <= max(2, 1e-5 * pairs), (mism, pairs)
