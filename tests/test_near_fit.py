"""The mixed path's near-field factor (host fit, no GPU): g(q) = (1 - e^-q)/q
of Eq. 8 with q = kappa rho^2 is evaluated by the FP32 kernels as a
polynomial in rho^2 (Horner with fused multiply-adds) over the near pairs'
range, or up to q = 1 with the exponential form beyond.  Evaluated here the
way the kernels do (FP32 coefficients, one rounding per FMA) against the
closed form (expm1 in FP64), the fit stays within the requested tolerance
plus FP32 rounding over its whole range, and the switch to the exponential
form happens exactly when the near pairs reach beyond q = 2."""
import numpy as np
import pytest

import __graft_entry__


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    from paper_0905_2637_gb300 import _lib
    return _lib


def horner_fma32(coef, deg, s):
    """coef[deg] s^deg + ... in FP32 with one rounding per step (an FP32
    product is exact in FP64, so fl32(v s + a) is the fused result)."""
    v = np.full(s.shape, coef[deg], np.float32)
    for k in range(deg - 1, -1, -1):
        v = (v.astype(np.float64) * s.astype(np.float64) + np.float64(coef[k])).astype(np.float32)
    return v.astype(np.float64)


CASES = [
    (0.002, 1 / 1024),          # clustered-16M: sigma about two leaf widths
    (0.004, 1 / 512),           # clustered-4M
    (1.5 / 1024, 1 / 256),      # lattice-1M
    (0.5 / np.sqrt(40_000), 1 / 64),   # a batch tree: sigma well below the leaf
    (0.02, 1 / 1024),           # Lamb-Oseen: many leaves per sigma
    (1e-4, 1 / 8),              # extreme: q up to 1e6 in the near field
]


@pytest.mark.parametrize("tol", [1e-7, 2.5e-6, 1e-5])
@pytest.mark.parametrize("sigma,w", CASES)
def test_polynomial_within_tolerance_in_fp32(lib, sigma, w, tol):
    f = lib.petfmm_debug_near_fit(sigma, w, tol)
    kappa = w * w / (2 * sigma * sigma)
    assert f["kappa"] == float(np.float32(kappa))
    rho2max = 8.0 * (1.0 + 1e-6)          # near pairs: at most 2 leaf widths per axis
    general = kappa * rho2max > 2.0
    assert f["general"] == int(general)
    assert 4 <= f["deg"] <= 12
    assert not np.any(f["coef"][f["deg"] + 1:])
    split = f["split_rho2"]
    assert split == float(np.float32(1.0 / kappa if general else rho2max))
    coef = f["coef"].astype(np.float32)
    s = np.linspace(0.0, split, 40_001).astype(np.float32)
    q = np.float64(np.float32(kappa)) * s.astype(np.float64)
    g = np.where(q > 0, -np.expm1(-q) / np.where(q > 0, q, 1.0), 1.0)
    err = np.max(np.abs(horner_fma32(coef, f["deg"], s) - g) / g)
    assert err <= tol + 2e-7, (err, f["deg"])


def test_a_wrong_coefficient_order_fails(lib):
    # the check above is sharp enough to see a transposed or mis-scaled fit
    f = lib.petfmm_debug_near_fit(0.002, 1 / 1024, 2.5e-6)
    coef = f["coef"].astype(np.float32)
    s = np.linspace(0.0, f["split_rho2"], 2001).astype(np.float32)
    q = np.float64(np.float32(f["kappa"])) * s.astype(np.float64)
    g = np.where(q > 0, -np.expm1(-q) / np.where(q > 0, q, 1.0), 1.0)
    rev = np.zeros_like(coef)
    rev[:f["deg"] + 1] = coef[:f["deg"] + 1][::-1]
    assert np.max(np.abs(horner_fma32(rev, f["deg"], s) - g) / g) > 1e-2
    half = coef * np.float32(0.5) ** np.arange(coef.size, dtype=np.float32)
    assert np.max(np.abs(horner_fma32(half, f["deg"], s) - g) / g) > 1e-3


def test_bad_arguments(lib):
    for args in ((0.0, 0.1, 1e-6), (0.1, 0.0, 1e-6), (0.1, 0.1, 0.0)):
        with pytest.raises(lib.PetfmmError):
            lib.petfmm_debug_near_fit(*args)
