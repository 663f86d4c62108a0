"""The accept decision of the collision kernels (Eq. proba3: a pair collides
if U < p), through pcc_accept_check, against the oracle's: U is compared
with p digit by digit, and the 48-bit rest is drawn only on the tie of the
16-bit first digit, a = floor(2^16 p), which the collision steps reach with
probability 2^-16 per evaluated pair.  Here two thirds of the digits are set
to the tie, so the rest branch runs thousands of times, in FP64 (plain path)
and with p rounded to FP32 (batched path); both must equal the oracle
exactly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pcc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_02814_gb300 import build, pcc as p
    build.build()
    return p


def test_accept_decision_matches_oracle(pcc, orc):
    rng = np.random.default_rng(17)
    n = 6000
    step, seed = 123456, 0x0BADC0DE12345678
    # probabilities from 1e-15 to 1 (log-uniform), plus exact edges
    p = 10.0 ** rng.uniform(-15.0, 0.0, n)
    p[:5] = [0.0, 1.0, 2.0 ** -32, 1.0 - 2.0 ** -40, 2.0 ** -16]
    p32 = p.astype(np.float32).astype(np.float64)
    r = rng.integers(0, 2 ** 16, n, dtype=np.uint64)
    tie64 = np.minimum(np.floor(p * 2.0 ** 16), 2 ** 16 - 1).astype(np.uint64)
    tie32 = np.minimum(np.floor(p32 * 2.0 ** 16), 2 ** 16 - 1).astype(np.uint64)
    r[0::3] = tie64[0::3]
    r[1::3] = tie32[1::3]
    c0 = rng.integers(0, 2 ** 20, n, dtype=np.uint64)
    cell = rng.integers(0, 2 ** 24, n, dtype=np.uint64)
    tag = (rng.integers(0, 3, n) | (6 << 4) | (rng.integers(0, 4, n) << 8)).astype(np.uint64)

    def dev32(a):
        return torch.as_tensor(a.astype(np.uint32).view(np.int32), device="cuda")

    o32, o64 = pcc.accept_check(dev32(r), torch.as_tensor(p, device="cuda"), dev32(c0), dev32(cell), dev32(tag),
                                step, seed)
    o32, o64 = o32.cpu().numpy(), o64.cpu().numpy()
    ref64 = np.array([orc.accept(int(r[i]), float(p[i]), int(c0[i]), int(cell[i]), step, int(tag[i]), seed)
                      for i in range(n)])
    ref32 = np.array([orc.accept(int(r[i]), float(p32[i]), int(c0[i]), int(cell[i]), step, int(tag[i]), seed)
                      for i in range(n)])
    assert np.array_equal(o64, ref64.astype(np.int32))
    assert np.array_equal(o32, ref32.astype(np.int32))
    # the tie branch really ran, both ways
    ties = r == tie64
    assert ties.sum() > 1500 and 0 < ref64[ties].sum() < ties.sum()
    assert o64[0] == 0 and o64[1] == 1


def test_accept_check_rejects_bad_arrays(pcc):
    z = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(pcc.PccError):
        pcc.accept_check(z, torch.zeros(4, dtype=torch.float32, device="cuda"), z, z, z, 0, 0)
