"""The FP64 <-> FP32 conversions of the mixed-precision path (mgpbd_convert).

The library converts between its FP64 Krylov vectors and its FP32 V-cycle
with integer code (the hardware conversion issues on the narrow FP64 pipe).
Both directions must give exactly what IEEE 754 fixes: binary64 -> binary32
rounds to nearest with ties to even, binary32 -> binary64 is exact.  numpy's
astype on the host and torch's cast on the GPU serve as the two references.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def special_doubles():
    f32max = float(np.finfo(np.float32).max)
    tiny32 = float(np.finfo(np.float32).tiny)  # 2^-126
    sub32 = 2.0 ** -149
    v = [0.0, -0.0, np.inf, -np.inf, 1.0, -1.0, f32max, -f32max, tiny32, -tiny32, sub32, -sub32,
         sub32 / 2, sub32 * 0.75, sub32 * 1.5, sub32 * 2.5, sub32 / 2 * (1 + 2 ** -52),
         tiny32 * (1 - 2 ** -24), tiny32 * (1 - 2 ** -25), 2.0 ** 128, 2.0 ** 127 * (2 - 2 ** -24),
         2.0 ** 127 * (2 - 2 ** -25), 2.0 ** 127 * (2 - 2 ** -23), 5e-324, -5e-324, 1e-310,
         1e300, -1e300, 2.0 ** -1074 * 3, 3.0e-39, 1.0e-45]
    out = list(v)
    # ties and near-ties at many exponents: 1 + k/2^24 with k odd or even
    for e in range(-140, 128, 7):
        for k in (1, 2, 3, 5, 6):
            base = 2.0 ** e
            out += [base * (1 + k * 2.0 ** -24), -base * (1 + k * 2.0 ** -24),
                    base * (1 + k * 2.0 ** -24 + 2.0 ** -50), base * (1 + k * 2.0 ** -24 - 2.0 ** -50)]
    return np.array(out, dtype=np.float64)


def run_convert(in64=None, in32=None):
    from paper_2505_13390_gb300.mgpbd import convert
    d64 = torch.from_numpy(in64).cuda() if in64 is not None else None
    d32 = torch.from_numpy(in32).cuda() if in32 is not None else None
    o32 = torch.empty(d64.numel(), dtype=torch.float32, device="cuda") if d64 is not None else None
    o64 = torch.empty(d32.numel(), dtype=torch.float64, device="cuda") if d32 is not None else None
    convert(d64, o32, d32, o64)
    torch.cuda.synchronize()
    return (o32.cpu().numpy() if o32 is not None else None,
            o64.cpu().numpy() if o64 is not None else None, d64, d32)


def same_bits(a, b):
    nan_a, nan_b = np.isnan(a), np.isnan(b)
    assert np.array_equal(nan_a, nan_b)
    ia = a[~nan_a].view(np.uint32 if a.dtype == np.float32 else np.uint64)
    ib = b[~nan_b].view(np.uint32 if b.dtype == np.float32 else np.uint64)
    bad = np.nonzero(ia != ib)[0]
    assert bad.size == 0, (a[~nan_a][bad[:5]], b[~nan_b][bad[:5]])


def test_narrow_rounds_to_nearest_even():
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 2 ** 64, size=1 << 20, dtype=np.uint64)
    # bias half of the patterns into the binary32 range (exponents 896..1151)
    e = rng.integers(860, 1160, size=bits.size // 2).astype(np.uint64)
    bits[: bits.size // 2] = (bits[: bits.size // 2] & ~np.uint64(0x7FF << 52)) | (e << np.uint64(52))
    x = np.concatenate([bits.view(np.float64), special_doubles()])
    with np.errstate(over="ignore"):
        want = x.astype(np.float32)
    got, _, d64, _ = run_convert(in64=x)
    same_bits(got, want)
    same_bits(got, d64.to(torch.float32).cpu().numpy())


def test_widen_is_exact():
    rng = np.random.default_rng(12)
    bits = rng.integers(0, 2 ** 32, size=1 << 20, dtype=np.uint64).astype(np.uint32)
    extra = np.array([0, 0x80000000, 1, 0x80000001, 0x007FFFFF, 0x00400000, 0x00800000, 0x7F7FFFFF,
                      0x7F800000, 0xFF800000, 0x3F800000, 0x00000003], dtype=np.uint32)
    x = np.concatenate([bits, extra]).view(np.float32)
    _, got, _, d32 = run_convert(in32=x)
    same_bits(got, x.astype(np.float64))
    same_bits(got, d32.to(torch.float64).cpu().numpy())


def test_rejects_bad_arguments():
    from paper_2505_13390_gb300 import mgpbd
    lib = mgpbd.load()
    a = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert lib.mgpbd_convert(None, None, None, None, -1, None) == mgpbd.E_INVALID
    assert lib.mgpbd_convert(a.data_ptr(), None, None, None, 4, None) == mgpbd.E_INVALID
    assert lib.mgpbd_convert(None, None, None, None, 0, None) == mgpbd.OK
