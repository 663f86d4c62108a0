"""The allocation-free totals entry point, for callers that may not allocate
device memory while they run (a simulation that sizes all its buffers at
start-up, an application whose own allocator owns the device).  It gives
the same sums as pcc_totals on two calls in a row that share its fixed
scratch, also at exactly its cell limit; a call changes neither the
device's free memory nor torch's reserved memory; and cell counts beyond
the limit are rejected.  Collected last so that a failure here stops a run
only after every other test has run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

MAX_CELLS = 4_194_304


def _ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_02814_gb300 import build, pcc
    build.build()
    return pcc


def test_totals_noalloc_matches_pcc_totals():
    pcc = _ready()
    from paper_1907_02814_gb300 import workloads as W
    ctx = pcc.Context(0)
    rng = np.random.default_rng(21)
    results = []
    for call, (n_cells, seed) in enumerate(((3000, 5), (1500, 6))):
        wl = W.solid_cu(n_cells=n_cells, e_per_cell=rng.integers(0, 40, n_cells), i_per_cell=3, seed=seed,
                        photons_per_cell=rng.integers(0, 9, n_cells))
        for name in ("em", "ph"):
            d = wl.species[name]
            n = len(d["w"])
            sp = pcc.DeviceSpecies.empty(n_cells, n + int(0.1 * n) + 3 * n_cells)
            pcc.bin(ctx, pcc.particles_to_device(d), n_cells, sp, slack_abs=1, slack_rel=0.1)
            ref = pcc.totals(ctx, n_cells, sp, is_photon=(name == "ph"))
            out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            pcc.totals_noalloc(n_cells, sp, out, is_photon=(name == "ph"))
            torch.cuda.synchronize()
            np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12)
            results.append(out.cpu().numpy())
    assert len(results) == 4 and all(np.all(np.isfinite(r)) and r[0] > 0 for r in results)

    # a further call allocates nothing, on the device or in torch's allocator
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    pcc.totals_noalloc(n_cells, sp, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0

    # beyond the fixed scratch: a clear error, nothing launched
    with pytest.raises(pcc.PccError, match="exceed the fixed scratch limit"):
        pcc.totals_noalloc(MAX_CELLS + 1, sp, out)
    ctx.close()


def test_totals_noalloc_at_the_cell_limit():
    """Exactly 4,194,304 cells (every block of the fixed scratch in use),
    with particles in the first, a middle and the last cell."""
    pcc = _ready()
    ctx = pcc.Context(0)
    rng = np.random.default_rng(4)
    cells = np.array([0] * 5 + [MAX_CELLS // 2] * 3 + [MAX_CELLS - 1] * 7, dtype=np.int32)
    n = len(cells)
    d = {"ux": rng.normal(size=n).astype(np.float32), "uy": rng.normal(size=n).astype(np.float32),
         "uz": rng.normal(size=n).astype(np.float32), "w": rng.uniform(1.0, 2.0, n).astype(np.float32),
         "pid": np.arange(n, dtype=np.uint64), "cell": cells, "x": None}
    sp = pcc.DeviceSpecies.empty(MAX_CELLS, n + MAX_CELLS)
    pcc.bin(ctx, pcc.particles_to_device(d), MAX_CELLS, sp, slack_abs=1, slack_rel=0.0)
    ref = pcc.totals(ctx, MAX_CELLS, sp)
    for _ in range(2):
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        pcc.totals_noalloc(MAX_CELLS, sp, out)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12)
    u = np.sqrt(d["ux"].astype(np.float64) ** 2 + d["uy"].astype(np.float64) ** 2 + d["uz"].astype(np.float64) ** 2)
    w = d["w"].astype(np.float64)
    np.testing.assert_allclose(out.cpu().numpy(), [w.sum(), (w * np.sqrt(1 + u * u)).sum(), (w * u).sum()],
                               rtol=1e-12)
    ctx.close()
