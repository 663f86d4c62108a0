"""The Au foil workload with transport: each step is collide (Brems + BH),
commit, a free-streaming push with reflecting walls, and a re-bin of every
species by cell.  The push is test harness (the pusher is not part of the
collision method); it is the same float32 operation sequence on both sides,
so the FP64 GPU path must stay identical to the oracle over several steps
with 31 material tables (Z* = 10..40) and positions carried through."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1907_02814_gb300 import workloads as W  # noqa: E402

C_LIGHT = np.float32(299792458.0)
MASK = 1 | 4            # Brems + Bethe-Heitler


@pytest.fixture(scope="module")
def pcc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_02814_gb300 import build, pcc as p
    build.build()
    return p


def push_np(d, n, dt, dx, n_cells, photon):
    """x += v dt (float32), reflect at 0 and L, cell = floor(x / dx)."""
    ux, uy, uz, x = d["ux"][:n], d["uy"][:n], d["uz"][:n], d["x"][:n]
    u2 = ux * ux + uy * uy + uz * uz
    norm = np.sqrt(u2) if photon else np.sqrt(np.float32(1.0) + u2)
    xn = x + (ux / norm) * C_LIGHT * np.float32(dt)
    L = np.float32(dx * n_cells)
    lo, hi = xn < 0, xn > L
    xn = np.where(lo, -xn, np.where(hi, L + L - xn, xn)).astype(np.float32)
    d["ux"][:n] = np.where(lo | hi, -ux, ux)
    d["x"][:n] = xn
    d["cell"][:n] = np.clip(np.floor(xn / np.float32(dx)), 0, n_cells - 1).astype(np.int32)


def push_torch(t, dt, dx, n_cells, photon):
    ux, uy, uz, x = t["ux"], t["uy"], t["uz"], t["x"]
    u2 = ux * ux + uy * uy + uz * uz
    norm = torch.sqrt(u2) if photon else torch.sqrt(1.0 + u2)
    xn = x + (ux / norm) * float(C_LIGHT) * np.float32(dt).item()
    L = np.float32(dx * n_cells).item()
    lo, hi = xn < 0, xn > L
    xn = torch.where(lo, -xn, torch.where(hi, (L + L) - xn, xn))
    t["ux"] = torch.where(lo | hi, -ux, ux)
    t["x"] = xn
    t["cell"] = torch.clamp(torch.floor(xn / np.float32(dx).item()), 0, n_cells - 1).to(torch.int32)


def live_flat(sp):
    """Live particles of a DeviceSpecies as flat tensors (storage order)."""
    cnt = sp.cell_count.long()
    n_cells = cnt.numel()
    cell = torch.repeat_interleave(torch.arange(n_cells, device=cnt.device), cnt)
    first = torch.repeat_interleave(sp.cell_start[:-1].long(), cnt)
    run0 = torch.cumsum(cnt, 0) - cnt
    idx = first + (torch.arange(int(cnt.sum()), device=cnt.device) - torch.repeat_interleave(run0, cnt))
    return {"ux": sp.ux[idx], "uy": sp.uy[idx], "uz": sp.uz[idx], "w": sp.w[idx], "pid": sp.pid[idx],
            "x": sp.x[idx], "cell": cell.to(torch.int32), "n": int(cnt.sum())}


def rebin(pcc, ctx, t, n_cells, slack):
    sp = pcc.DeviceSpecies.empty(n_cells, t["n"] + (slack + 1) * n_cells, with_x=True)
    pcc.bin(ctx, t, n_cells, sp, slack_abs=slack, slack_rel=0.0)
    return sp


def run_gpu(pcc, ctx, wl, steps, precision, slack=64):
    mats = [pcc.material(m.Z, m.Zstar, m.n_i, m.T_e) for m in wl.materials]
    ctx.tables_build(mats, pcc.table_spec(n_rows=96, n_cols=96))
    mat = torch.as_tensor(wl.material_of_cell, device="cuda")
    dev = {}
    for k, d in wl.species.items():
        dev[k] = rebin(pcc, ctx, pcc.particles_to_device(d) if len(d["w"]) else
                       {"n": 0, "ux": None, "uy": None, "uz": None, "w": None, "pid": None, "cell": None,
                        "x": torch.zeros(0, device="cuda")}, wl.n_cells, slack)
    ctx.read_status()
    status, stats = 0, []
    for s in range(steps):
        pcc.collide(ctx, wl.n_cells, mat, wl.ion_mass, dev["em"], dev["ep"], dev["ph"], dev["ion"], wl.dt, wl.seed,
                    s, mask=MASK, precision=precision)
        for k in ("em", "ep", "ph"):
            pcc.append_secondaries(ctx, wl.n_cells, dev[k])
        st, sts = ctx.read_status()
        status |= st
        stats.append(sts)
        for k in ("em", "ep", "ph", "ion"):
            t = live_flat(dev[k])
            if t["n"]:
                push_torch(t, wl.dt, wl.dx, wl.n_cells, k == "ph")
            dev[k] = rebin(pcc, ctx, t, wl.n_cells, slack)
    return dev, status, stats


def test_foil_transport_matches_oracle(pcc, orc):
    wl = W.au_foil(n_cells=192, mean_e=40, i_per_cell=12, dt=40e-15, dx=10e-6)
    steps = 4
    ctx = pcc.Context(0)
    dev, status, stats = run_gpu(pcc, ctx, wl, steps, pcc.FP64_PLAIN)
    ctx.close()
    T = orc.OracleTables([orc.material(m.Z, m.Zstar, m.n_i, m.T_e) for m in wl.materials],
                         orc.table_spec(n_rows=96, n_cols=96))
    sp = {k: orc.OracleSpecies(v, cap=len(v["w"]) + 100000) for k, v in wl.species.items()}
    for s in range(steps):
        _, st = orc.step(T, wl.n_cells, wl.material_of_cell, sp["em"], sp["ep"], sp["ph"], sp["ion"], wl.ion_mass,
                         wl.dt, wl.seed, s, mask=MASK)
        assert st["rc"] == 0
        assert stats[s]["pairs"] == [int(v) for v in st["pairs"]], s
        assert stats[s]["created"] == [int(v) for v in st["created"]], s
        for k in ("em", "ep", "ph", "ion"):
            o = sp[k]
            d = {"ux": o.ux, "uy": o.uy, "uz": o.uz, "x": o.x, "cell": o.cell}
            if o.n:
                push_np(d, o.n, wl.dt, wl.dx, wl.n_cells, k == "ph")
    assert sum(sum(s_["created"]) for s_ in stats) > 20
    assert status & pcc.ST_CAPACITY == 0
    for k in ("em", "ep", "ph", "ion"):
        g, c = dev[k].live_host(), sp[k].canonical()
        assert np.array_equal(g["pid"], c["pid"]), k
        assert np.array_equal(g["cell"], c["cell"]), k
        for f in ("ux", "uy", "uz", "x"):
            np.testing.assert_allclose(g[f], c[f], rtol=2e-6, atol=1e-6, err_msg=f"{k}.{f}")


def test_foil_full_size_100_steps(pcc):
    """16384 cells, Poisson(256) electrons (about 4.2e6), 31 materials, 100
    steps of collide + push + re-bin on the batched FP32 path: no overflow,
    charge conserved to the last bit of the weights' sum."""
    wl = W.au_foil(dt=40e-15, dx=10e-6)
    ctx = pcc.Context(0)
    dev, status, stats = run_gpu(pcc, ctx, wl, 100, pcc.FP32_BATCHED, slack=128)
    q = float(pcc.totals(ctx, wl.n_cells, dev["ep"])[0]) - float(pcc.totals(ctx, wl.n_cells, dev["em"])[0])
    ctx.close()
    q0 = -float(np.sum(wl.species["em"]["w"].astype(np.float64)))
    assert status & (pcc.ST_CAPACITY | pcc.ST_NONFINITE | pcc.ST_TIMEOUT) == 0, status
    assert sum(s["pairs"][0] for s in stats) >= 100 * 4_000_000
    assert sum(s["created"][4] for s in stats) > 0 and sum(s["created"][0] for s in stats) > 1000
    assert abs(q - q0) <= 1e-12 * abs(q0)
