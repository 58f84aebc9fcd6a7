"""The integer-operation conversions of the FP64 residual (double -> float,
round to nearest even) and of the mixed path's FP64 update (float -> double)
equal the hardware conversions bit for bit (IEEE 754 roundTiesToEven), on
random bit patterns over every exponent and on the cases where a rounding
rule decides: ties, one double ulp either side of a tie, carries out of the
fraction, the overflow threshold, the edge of the normal float range,
zeros, infinities and NaNs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _doubles(rng):
    parts = [rng.integers(0, 2**64, size=1 << 20, dtype=np.uint64).view(np.float64)]
    # every float exponent, random fractions
    parts.append(rng.uniform(-1, 1, 1 << 18) * np.exp2(rng.integers(-160, 140, 1 << 18)))
    # ties between neighbouring floats, and one double ulp either side
    fl = rng.integers(0, 2**32, size=1 << 18, dtype=np.uint64).astype(np.uint32).view(np.float32)
    fl = fl[np.isfinite(fl)]
    nxt = np.nextafter(fl, np.float32(np.inf), dtype=np.float32)
    ok = np.isfinite(nxt)
    mid = (fl[ok].astype(np.float64) + nxt[ok].astype(np.float64)) / 2
    parts += [mid, np.nextafter(mid, np.inf), np.nextafter(mid, -np.inf)]
    # carries out of the fraction: just below powers of two
    p2 = np.exp2(np.arange(-149, 129, dtype=np.float64))
    parts += [np.nextafter(p2, 0.0), -np.nextafter(p2, 0.0), p2, -p2]
    fmax = float(np.finfo(np.float32).max)
    half_ulp = 2.0 ** (127 - 24)
    tiny = float(np.finfo(np.float32).tiny)
    special = [0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax, fmax + half_ulp, np.nextafter(fmax + half_ulp, 0.0),
               np.nextafter(fmax + half_ulp, np.inf), tiny, -tiny, np.nextafter(tiny, 0.0), tiny / 2, 5e-324, 1e308]
    parts.append(np.array(special, dtype=np.float64))
    return np.concatenate(parts)


def test_conversions_equal_the_hardware_bit_for_bit():
    import torch
    import paper_2205_09411_gb300 as G
    rng = np.random.default_rng(20220519)
    x = _doubles(rng)
    f = rng.integers(0, 2**32, size=x.size, dtype=np.uint64).astype(np.uint32).view(np.float32)
    f[:8] = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-40, np.finfo(np.float32).tiny], dtype=np.float32)
    dx = torch.from_numpy(x).cuda()
    df = torch.from_numpy(f.copy()).cuda()
    bad = torch.zeros(2, dtype=torch.int64, device="cuda")
    G.selftest_conversions(dx, df, bad)
    torch.cuda.synchronize()
    assert bad.cpu().tolist() == [0, 0]
