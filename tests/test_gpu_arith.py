"""The pair arithmetic of each precision mode, element by element (steps
a1-a3 of one pair, Sec. III-IV), against exact references in extended
precision:
  - the FP32 hardware 1/sqrt seed over every float in [1, 4) (the seed's
    error is periodic in exponent pairs, so this covers all normal inputs);
  - each mode's r^-3 over displacements spanning twelve decades, with the
    error each mode's arithmetic allows."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

# worst relative error of r^-3 by mode (measured values well inside):
#   fp64: third-order correction of a compensated FP32 residual, about 2^-42;
#   df64: double-float r^2 and residual, about 2^-44 plus the final sum;
#   sqrtdiv and two Newton steps: FP64 rounding (a few ulp);
#   one Newton step squares the seed error (1.5 e^2, times 3 for the cube);
#   the bare seed: 3 x 2^-22; mixed: FP32 rounding of d and the corrected bulk;
#   mixed_split_rsq: the bare seed cubed in FP32 (3 x 2^-22.9 = 3.7e-7) plus
#   the FP32 rounding of d, r^2 and the cube.
BOUND = {"fp64": 4e-13, "df64": 2e-13, "sqrtdiv": 2e-15, "rsq_nr2": 2e-15, "rsq_nr1": 1e-12,
         "rsq": 1e-6, "mixed": 1e-6, "mixed_split": 1e-6, "mixed_split_rsq": 7e-7}


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_11143_gb300 as nbm
    nbm.lib()
    return nbm


def test_rsqrt_seed_exhaustive_on_1_to_4(nb):
    bits = np.arange(np.float32(1.0).view(np.uint32), np.float32(4.0).view(np.uint32), dtype=np.uint32)
    x = bits.view(np.float32)
    y = nb.rsqrt_seed_probe(torch.from_numpy(x)).cpu().numpy().astype(np.float64)
    ref = 1.0 / np.sqrt(x.astype(np.float64))
    err = np.abs(y / ref - 1.0)
    print("seed: %d inputs, max rel err %.3e = 2^%.2f" % (x.size, err.max(), np.log2(err.max())))
    assert x.size == 1 << 24
    assert err.max() <= 2.0 ** -22


def displacements(n, seed):
    rng = np.random.default_rng(seed)
    mag = 10.0 ** rng.uniform(-9.0, 3.0, n)  # 1 nm to 1 km
    u = rng.standard_normal((3, n))
    u /= np.linalg.norm(u, axis=0)
    d = u * mag
    # exponent edges of r^2: |d| on either side of powers of two, inside the
    # FP32 modes' range (|d| >= 2^-40 never meets their overflow clamp)
    k = np.arange(-36, 10)
    edge = np.concatenate([2.0 ** k * (1 + 2.0 ** -52), 2.0 ** k * (1 - 2.0 ** -53), 2.0 ** (k + 0.5)])
    e = np.zeros((3, edge.size))
    e[0] = edge
    return np.concatenate([d, e], axis=1)


def exact_rinv3(d, soft2=0.0):
    dl = d.astype(np.longdouble)
    r2 = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2] + np.longdouble(soft2)
    return r2 ** np.longdouble(-1.5)


@pytest.mark.parametrize("precision", list(BOUND))
def test_rinv3_by_mode(nb, precision):
    d = displacements(1 << 21, 3)
    ref = exact_rinv3(d)
    got = nb.rinv3_probe(precision, d).cpu().numpy()
    err = np.abs((got.astype(np.longdouble) - ref) / ref).astype(np.float64)
    print("%s: max %.3e  mean %.3e" % (precision, err.max(), err.mean()))
    assert np.all(np.isfinite(got))
    assert err.max() <= BOUND[precision]


@pytest.mark.parametrize("precision", ["fp64", "sqrtdiv", "rsq_nr1", "rsq_nr2"])
def test_rinv3_fp64_modes_full_exponent_range(nb, precision):
    """FP64 modes over every r^2 exponent whose r^-3 is a normal double
    (|d| from 2^-330 to 2^330), where the FP32 seed works on the
    exponent-reduced significand."""
    rng = np.random.default_rng(5)
    n = 1 << 18
    mag = 2.0 ** rng.uniform(-330.0, 330.0, n)
    u = rng.standard_normal((3, n))
    u /= np.linalg.norm(u, axis=0)
    d = u * mag
    ref = exact_rinv3(d)
    got = nb.rinv3_probe(precision, d).cpu().numpy()
    err = np.abs((got.astype(np.longdouble) - ref) / ref).astype(np.float64)
    print("%s: max %.3e" % (precision, err.max()))
    assert err.max() <= BOUND[precision]


def test_rinv3_softening_and_zero(nb):
    d = displacements(1 << 16, 4) * 1e-6
    soft2 = (0.3e-6) ** 2
    ref = exact_rinv3(d, soft2)
    for prec in ("fp64", "df64", "mixed"):
        got = nb.rinv3_probe(prec, d, soft2=soft2).cpu().numpy()
        err = np.abs((got.astype(np.longdouble) - ref) / ref).astype(np.float64)
        assert err.max() <= BOUND[prec], (prec, err.max())
    z = np.zeros((3, 4))
    for prec in ("fp64", "sqrtdiv", "rsq", "rsq_nr1", "rsq_nr2"):
        assert np.all(nb.rinv3_probe(prec, z).cpu().numpy() == 0.0), prec
    for prec in ("df64", "mixed", "mixed_split", "mixed_split_rsq"):  # clamped seed, finite: d * s = 0
        assert np.all(np.isfinite(nb.rinv3_probe(prec, z).cpu().numpy())), prec


def test_probe_rejects_bad_arguments(nb):
    L = nb.lib()
    assert L.nb_rinv3_probe(99, 4, None, None, None, 0.0, None, None) == 1
    assert L.nb_rinv3_probe(0, -1, None, None, None, 0.0, None, None) == 1
    assert L.nb_rinv3_probe(0, 4, None, None, None, 0.0, None, None) == 1
    assert L.nb_rinv3_probe(0, 0, None, None, None, 0.0, None, None) == 0
    assert L.nb_rsqrt_seed_probe(-1, None, None, None) == 1
