"""Error of the FP64 kernels' reciprocal and reciprocal square root
(Newton-Raphson from a single-precision seed) against IEEE results."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2404_08247_gb300 import build as B
    B.build()
    from paper_2404_08247_gb300 import rhd
    rhd.load()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return rhd


def test_reciprocal_and_rsqrt_within_two_ulp(R):
    rng = np.random.default_rng(0)
    # log-uniform over 1e-300 .. 1e300: most inside the seed's float exponent
    # range, the rest through the IEEE fallback; plus edges of that range
    x = 10.0 ** rng.uniform(-300, 300, 400000)
    x = np.concatenate([x, 10.0 ** rng.uniform(-40, 40, 400000),
                        2.0 ** np.arange(-130.0, 131.0), [1.0, 3.0, 1e-36, 1e36]])
    xd = torch.from_numpy(x).cuda()
    r, q = R.eval_recip(xd)
    r = r.cpu().numpy()
    q = q.cpu().numpy()
    u = 2.0 ** -53  # unit roundoff
    rr = 1.0 / x             # correctly rounded
    qq = 1.0 / np.sqrt(x)    # two roundings
    rel_r = np.abs(r - rr) / rr
    rel_q = np.abs(q - qq) / qq
    assert np.isfinite(r).all() and np.isfinite(q).all()
    assert rel_r.max() <= 4 * u, rel_r.max()   # within 2 ulp of IEEE division
    assert rel_q.max() <= 6 * u, rel_q.max()   # within 3 ulp
