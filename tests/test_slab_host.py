"""Host side of the field-free slab study, on CPU tensors: the live-particle
gather of a cell-region species and the straight-line photon transport with
removal at the slab faces."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1907_02814_gb300 import slab  # noqa: E402

C = slab.C_LIGHT


def _species(start, count, n_slots):
    f = lambda: torch.arange(n_slots, dtype=torch.float32)
    return types.SimpleNamespace(cell_start=torch.tensor(start, dtype=torch.int32),
                                 cell_count=torch.tensor(count, dtype=torch.int32),
                                 ux=f(), uy=f() + 100, uz=f() + 200, w=f() + 300, x=f() + 400,
                                 pid=torch.arange(n_slots, dtype=torch.int64) + 1000)


def test_live_flat_gathers_the_live_slots_in_storage_order():
    # regions [0,4) [4,5) [5,9) with 2, 0 and 3 live particles
    sp = _species([0, 4, 5, 9], [2, 0, 3], 9)
    t = slab._live_flat(torch, sp)
    assert t["n"] == 5
    assert t["ux"].tolist() == [0, 1, 5, 6, 7]
    assert t["pid"].tolist() == [1000, 1001, 1005, 1006, 1007]
    assert t["cell"].tolist() == [0, 0, 2, 2, 2]
    assert t["w"].tolist() == [300, 301, 305, 306, 307]


def test_push_moves_at_c_and_removes_escaped_photons():
    dx, nx, dt = 1.0e-6, 4, 1.0e-15          # cells of 1 um, columns of 4 cells; c dt = 0.3 um
    ux = torch.tensor([1.0, -1.0, 0.0, 3.0, 1.0], dtype=torch.float32)
    uy = torch.tensor([0.0, 0.0, 2.0, 4.0, 0.0], dtype=torch.float32)
    x = torch.tensor([3.9e-6, 0.1e-6, 2.0e-6, 1.0e-6, 0.95e-6], dtype=torch.float32)
    t = {"ux": ux, "uy": uy, "uz": torch.zeros(5), "w": torch.ones(5), "pid": torch.arange(5),
         "x": x, "cell": torch.tensor([3, 4, 2, 5, 4], dtype=torch.int32)}     # cells 4, 5 are column 1
    out = slab._push_photons(torch, t, dt, dx, nx)
    # photon 0 leaves through the far face, photon 1 through the near one
    assert out["n"] == 3 and out["pid"].tolist() == [2, 3, 4]
    step = C * dt
    expect_x = np.array([2.0e-6, 1.0e-6 + 0.6 * step, 0.95e-6 + step])    # 3/5 of c along x for (3, 4)
    assert np.allclose(out["x"].numpy(), expect_x, rtol=1e-6)
    # cells are recomputed within each photon's own column
    assert out["cell"].tolist() == [2, 4 + 1, 4 + 1]
