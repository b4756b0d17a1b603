"""The INT8 split's fixed-point step, compiled for the host from the kernel
header (paper_2303_04353_gb300/csrc/split_int8_device.cuh), against the
oracle's restatement (Sec. "FP64x2 in terms of INT8": every entry becomes
X = rne(hi 2^sh) + rne(lo 2^sh) before its digits are taken).

The kernel forms X from the words of the two doubles with funnel shifts and
a carry trick for the rounding; the oracle from exact rationals.  The cases
are the ones a slip in that word arithmetic would get wrong: every shift
amount from the rounding range through all three word offsets, ties at
every rounding position (odd and even quotients), subnormals, signed zeros,
values just below a power of two and mixed signs of hi and lo.  Needs nvcc
(no GPU): the header's arithmetic is host-callable."""
import os
import random
import shutil
import struct
import subprocess

import pytest

from oracle import cascade_int8 as c8

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2303_04353_gb300", "csrc", "split_int8_device.cuh")

DRIVER = r"""
#include <cstdio>
#include <cstring>
#include "%s"
int main() {
    unsigned long long bh, bl;
    int sh;
    while (std::scanf("%%llx %%llx %%d", &bh, &bl, &sh) == 3) {
        double hi, lo;
        std::memcpy(&hi, &bh, 8);
        std::memcpy(&lo, &bl, 8);
        bool finite = true;
        const unsigned __int128 y = (unsigned __int128)ddg::split8::fixed_sum(hi, lo, sh, 0, finite);
        std::printf("%%016llx%%016llx %%d\n", (unsigned long long)(y >> 64),
                    (unsigned long long)y, finite ? 1 : 0);
    }
    return 0;
}
"""


def bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("fixed_point")
    src, exe = d / "driver.cu", d / "driver"
    src.write_text(DRIVER % HEADER)
    subprocess.run([nvcc, "-std=c++17", "-O1", "-x", "cu", str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    return str(exe)


def run(exe, cases):
    text = "".join(f"{bits(h):x} {bits(lo):x} {sh}\n" for h, lo, sh in cases)
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
    res = []
    for line in out.split():
        res.append(line)
    return [(int(res[i], 16), int(res[i + 1])) for i in range(0, len(res), 2)]


def in_range(x: float, sh: int) -> bool:
    """The form's range: |x| 2^sh < 2^74 (beyond it the kernel gives 0, an
    entry far above its block's max |hi|)."""
    if x == 0.0:
        return True
    _, e = __import__("math").frexp(x)
    return e + sh <= 74


def cases():
    rng = random.Random(7)
    out = []
    specials = [0.0, -0.0, 1.0, -1.0, 0.5, 5e-324, -5e-324, 2.2250738585072014e-308,
                2.225073858507201e-308, 1.0000000000000002, 0.9999999999999999, 3.0, -3.0,
                1.5, 2.0 ** -53, 1.5 * 2.0 ** -53, -(2.0 ** -60)]
    for hi in specials:
        for lo in specials:
            for sh in (-1100, -60, -54, -53, -52, -1, 0, 1, 10, 31, 32, 33, 52, 63, 64, 65, 72, 73,
                       1074, 1080, 1100, 1126):
                out.append((hi, lo, sh))
    # every rounding position with a tie, odd and even quotients
    for r in range(1, 64):
        for q in range(8):
            m = (1 << 52) | (q << (r if r < 52 else 0))
            if r <= 52:
                m |= 1 << (r - 1)            # exactly half of the unit at position r
            x = float(m) * 2.0 ** -52
            out.append((x, -x * 2.0 ** -60, 52 - r))
            out.append((-x, x * 2.0 ** -57, 52 - r))
    # random significands at every shift amount of hi and of lo
    for _ in range(4000):
        e = rng.randint(-1000, 1000)
        hi = rng.uniform(0.5, 1.0) * 2.0 ** (e - rng.randint(0, 70)) * rng.choice((-1, 1))
        lo = hi * 2.0 ** (-53 - rng.randint(0, 20)) * rng.uniform(-0.5, 0.5)
        out.append((hi, lo, 111 - e + rng.randint(-3, 3)))
    return [(h, lo, sh) for h, lo, sh in out if in_range(h, sh) and in_range(lo, sh)]


def test_fixed_sum_matches_the_oracle(driver):
    cs = cases()
    assert len(cs) > 8000
    got = run(driver, cs)
    for (h, lo, sh), (y, finite) in zip(cs, got):
        want = (c8.rne_scaled(h, sh) + c8.rne_scaled(lo, sh)) % (1 << 128)
        assert finite == 1
        assert y == want, (h, lo, sh)


def test_non_finite_entries_are_flagged(driver):
    inf, nan = float("inf"), float("nan")
    got = run(driver, [(inf, 0.0, 10), (1.0, nan, 10), (-inf, 1.0, 0), (1.0, 0.0, 10)])
    assert [f for _, f in got] == [0, 0, 0, 1]
