"""The corrector's division by the constants 6, 24 and 120 (Sec. 2's
r1, v1 and the predictor's j/6) takes one product and one FMA correction
with the correctly rounded reciprocal (Markstein's FMA division) instead of
a general IEEE division; the corrector is bit-exact to the oracle only if
that gives RN(a / b) for every a.  This checks the identity on random
doubles over a wide exponent range, in C on the host (gcc's fma is exact).
"""
import os
import shutil
import subprocess
import tempfile

import pytest

SRC = r"""
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>
static uint64_t s = 0x9E3779B97F4A7C15ull;
static uint64_t nxt(void) { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; }
int main(void) {
    const double bs[3] = {6.0, 24.0, 120.0};
    long long bad = 0;
    for (int k = 0; k < 3; ++k) {
        const double b = bs[k], y = 1.0 / b;
        for (long long t = 0; t < 2000000LL; ++t) {
            uint64_t u = nxt();
            uint64_t mant = u & 0x000FFFFFFFFFFFFFull;
            int e = (int)((u >> 52) % 241) - 120;
            uint64_t bits = ((uint64_t)(1023 + e) << 52) | mant | ((u & 1ull) << 63);
            double a;
            memcpy(&a, &bits, 8);
            const double q0 = a * y;
            const double r = fma(-q0, b, a);
            const double q1 = fma(r, y, q0);
            if (q1 != a / b) ++bad;
        }
    }
    printf("%lld\n", bad);
    return 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_fma_division_by_constants_is_correctly_rounded():
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "div.c")
        exe = os.path.join(d, "div")
        with open(src, "w") as f:
            f.write(SRC)
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-o", exe, src, "-lm"], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    assert int(out.strip()) == 0
