"""The allocation-free totals entry point (for callers that may not allocate
device memory during their run) gives the same sums as pcc_totals, on two
calls in a row that share its fixed scratch, and rejects cell counts beyond
its fixed limit.  Collected last so that a failure here stops a run only
after every other test has run."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_totals_noalloc_matches_pcc_totals():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_02814_gb300 import build, pcc
    from paper_1907_02814_gb300 import workloads as W
    build.build()
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
    # beyond the fixed scratch: a clear error, nothing launched
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(pcc.PccError, match="exceed the fixed scratch limit"):
        pcc.totals_noalloc(4_194_305, sp, out)
    ctx.close()
