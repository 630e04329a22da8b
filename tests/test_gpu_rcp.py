"""The library's double reciprocals (a single-precision seed refined by Newton-Raphson
steps, or by one third-order step in the near-field form, used
for 1/|xi_j - xi_i|^2 at every near pair of the discretised double layer, Sec. 5, and
for the far-field conversions) against IEEE division on the host, over a log-spaced
sweep with random mantissas: within 2 units in the last place of double."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import dev, host, zeros  # noqa: E402
from paper_1306_0612_gb300 import lbfmm as L  # noqa: E402

pytestmark = pytest.mark.gpu

ULP = 2.0 ** -52


def _sweep(lo_exp, hi_exp, n, seed):
    rng = np.random.default_rng(seed)
    e = rng.uniform(lo_exp, hi_exp, n)
    m = rng.uniform(1.0, 2.0, n)
    a = np.ldexp(m, np.floor(e).astype(int))
    # mantissas at the edges of each binade, and exact powers of two
    edge = np.concatenate([np.ldexp(1.0, np.arange(lo_exp, hi_exp)),
                           np.nextafter(np.ldexp(1.0, np.arange(lo_exp + 1, hi_exp)), 0.0)])
    return np.concatenate([a, edge])


@pytest.mark.parametrize("variant,lo,hi", [(1, -126, 126), (0, -99, 99)])
def test_reciprocal_against_division(variant, lo, hi):
    a = _sweep(lo, hi, 200000, 7 + variant)
    out = zeros(len(a))
    L.lbf_selftest_rcp(variant, dev(a), out)
    got = host(out)
    ref = 1.0 / a
    rel = np.abs(got - ref) / ref
    assert np.all(np.isfinite(got))
    assert rel.max() <= 2 * ULP, (rel.max() / ULP, a[np.argmax(rel)])


def test_general_reciprocal_outside_its_seed_range_divides():
    a = np.array([1e-40, 3e-35, 2e33, 1e300, 5e-300, -7.0, -1e-31])
    out = zeros(len(a))
    L.lbf_selftest_rcp(0, dev(a), out)
    assert np.max(np.abs(host(out) * a - 1.0)) <= 2 * ULP


def test_near_field_reciprocal_of_the_self_pair_shift():
    """The self pair of the near field enters with |dz|^2 = 1e-30 (a shift that keeps
    its term 0 x finite): its reciprocal is finite and correct."""
    a = np.array([1e-30, 1e-30 + 1e-45, 2.5e-29])
    out = zeros(len(a))
    L.lbf_selftest_rcp(1, dev(a), out)
    got = host(out)
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got * a - 1.0)) <= 2 * ULP
