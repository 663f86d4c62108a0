"""Thin-target yields of the batched FP32 path through the C ABI: the
Bremsstrahlung check of Fig. valid_brem_tf (Eq. N_br_theo1) and its
Bethe-Heitler and Trident counterparts, at eight times the oracle tests'
statistics, for weight ratios W_i/W_p in {2, 1, 1/2}: the created weight must
match the analytic yield whatever the ratio."""
import math

import numpy as np
import pytest
from scipy import integrate

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1907_02814_gb300 import workloads as W  # noqa: E402

C_LIGHT = 299792458.0
MEC2_MEV = 0.51099895
N_CELLS, STEPS = 2048, 8


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


def quad(f, a, b):
    return integrate.quad(f, a, b, epsabs=0.0, epsrel=1e-11, limit=400)[0]


def run(pcc, ctx, wl, mask, steps=STEPS):
    ctx.tables_build([pcc.material(m.Z, m.Zstar, m.n_i, m.T_e) for m in wl.materials],
                     pcc.table_spec(n_rows=128, n_cols=128))
    dev = {}
    for name, d in wl.species.items():
        n = len(d["w"])
        sp = pcc.DeviceSpecies.empty(wl.n_cells, n + 64 * wl.n_cells + n // 4)
        if n:
            pcc.bin(ctx, pcc.particles_to_device(d), wl.n_cells, sp, slack_abs=64, slack_rel=0.25)
        else:
            pcc.bin(ctx, {"n": 0, "ux": None, "uy": None, "uz": None, "w": None, "pid": None, "cell": None},
                    wl.n_cells, sp, slack_abs=64, slack_rel=0.25)
        dev[name] = sp
    mat = torch.as_tensor(wl.material_of_cell, device="cuda")
    ctx.read_status()
    for s in range(steps):
        pcc.collide(ctx, wl.n_cells, mat, wl.ion_mass, dev["em"], dev["ep"], dev["ph"], dev["ion"], wl.dt, wl.seed,
                    s, mask=mask, precision=pcc.FP32_BATCHED)
        for k in ("em", "ep", "ph"):
            pcc.append_secondaries(ctx, wl.n_cells, dev[k])
    status, _ = ctx.read_status()
    assert status & (pcc.ST_CAPACITY | pcc.ST_NONFINITE | pcc.ST_TIMEOUT) == 0, status
    return dev


def created(dev, name):
    """Weight sum and count of the secondaries (id marker bit) of a species."""
    h = dev[name].live_host()
    sec = (h["pid"] >> np.uint64(63)) == 1
    return float(h["w"][sec].astype(np.float64).sum()), int(sec.sum()), h


def check(label, ratio, wsum, count, expected, slack):
    r = wsum / expected
    print(f"\n[thin target {label}, GPU FP32] W_i/W_p = {ratio}: yield / theory = {r:.4f} ({count} events)")
    assert count > 2000
    assert abs(r - 1.0) < 4.0 / math.sqrt(count) + slack, (label, ratio, r, count)


@pytest.mark.parametrize("ratio", [2.0, 1.0, 0.5])
def test_brems_thin_target(pcc, ctx, orc, ratio):
    g = 1.0 + 40.0 / MEC2_MEV
    v = C_LIGHT * math.sqrt(1.0 - 1.0 / g ** 2)
    dt = 150e-15
    wl = W.thin_target_beam(ratio, n_cells=N_CELLS, e_per_cell=64, seed=21, dt=dt)
    dev = run(pcc, ctx, wl, 1)
    wsum, count, _ = created(dev, "ph")
    s = orc.screening(orc.material(29, 0.0, 8e28, 0.0))
    T = g - 1.0
    sigma = quad(lambda lx: orc.dsdk_brems(s, g, math.exp(lx) * T) * T * math.exp(lx), math.log(1e-7), 0.0)
    check("Brems", ratio, wsum, count, 1e27 * 8e28 * v * sigma * STEPS * dt * N_CELLS, 0.01)


@pytest.mark.parametrize("ratio", [2.0, 1.0, 0.5])
def test_bethe_heitler_thin_target(pcc, ctx, orc, ratio):
    k = 100.0 / MEC2_MEV
    dt = 4e-13
    wl = W.thin_target_photon_beam(ratio, n_cells=N_CELLS, g_per_cell=64, seed=23, dt=dt)
    dev = run(pcc, ctx, wl, 4)
    wsum, count, _ = created(dev, "ep")
    s = orc.screening(orc.material(29, 0.0, 8e28, 0.0))
    sigma = quad(lambda gp: orc.dsdg_bh(s, k, gp), 1.0, k - 1.0)
    q = 8e28 * C_LIGHT * sigma * dt
    check("BH", ratio, wsum, count, 1e27 * (1.0 - (1.0 - q) ** STEPS) * N_CELLS, 0.01)
    # converted photons left the beam: the photon weight fell by the same amount
    ph = dev["ph"].live_host()
    assert float(ph["w"].astype(np.float64).sum()) == pytest.approx(1e27 * N_CELLS - wsum, rel=1e-5)


@pytest.mark.parametrize("ratio", [2.0, 1.0, 0.5])
def test_trident_thin_target(pcc, ctx, orc, ratio):
    """One long step: the created pairs join the projectiles only after it,
    so no cascade of secondary Tridents enters the count."""
    g = 1.0 + 500.0 / MEC2_MEV
    v = C_LIGHT * math.sqrt(1.0 - 1.0 / g ** 2)
    dt = 3.2e-11
    wl = W.thin_target_beam(ratio, n_cells=N_CELLS, e_per_cell=64, seed=24, dt=dt, gamma=g)
    dev = run(pcc, ctx, wl, 2, steps=1)
    wsum, count, _ = created(dev, "ep")
    check("Trident", ratio, wsum, count, 1e27 * 8e28 * v * orc.sigma_trident(29, g) * dt * N_CELLS, 0.01)
