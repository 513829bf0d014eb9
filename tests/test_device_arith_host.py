"""Host-side checks of the arithmetic helpers the kernels share
(csrc/apo_device.cuh): the division by a multiply-high used in the flat index
loops and for the mask sizes of Eq. 5, the Rastrigin cosine cos(2 pi v) by
exact reduction and a Taylor polynomial, and the Rosenbrock and Rastrigin terms
with explicit multiply-adds.  The helpers are compiled for the host by nvcc
(the same source and IEEE operations as on the device: exact integer
arithmetic, correctly rounded fmaf and rintf) and run without a GPU; the
references are plain integer division and the cosine in double precision."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_14982_gb300", "csrc")

PROGRAM = r"""
#include <cmath>
#include <cstdio>
#include <cstdint>
#include "apo_device.cuh"
using namespace apo;

static int fails = 0;
#define CHECK(c, ...) do { if (!(c)) { if (++fails < 20) { std::printf("FAIL " __VA_ARGS__); std::printf("\n"); } } } while (0)

static uint64_t lcg = 88172645463325252ull;
static uint32_t next32() { lcg ^= lcg << 13; lcg ^= lcg >> 7; lcg ^= lcg << 17; return (uint32_t)(lcg >> 16); }

int main()
{
    // floor(i / d) for i < 2^16: every i, d up to 1024 and a few larger d
    for (uint32_t d = 1; d <= 1024; ++d) {
        const uint32_t m = div_magic(d);
        for (uint32_t i = 0; i < 65536; ++i)
            if (div_small(i, m) != i / d) { CHECK(false, "div_small(%u, d %u)", i, d); break; }
    }
    for (uint32_t d : {1500u, 4095u, 4096u, 4097u, 28672u, 65535u}) {
        const uint32_t m = div_magic(d);
        for (uint32_t i = 0; i < 65536; ++i)
            if (div_small(i, m) != i / d) { CHECK(false, "div_small(%u, d %u)", i, d); break; }
    }
    // 64-bit reciprocal: any 32-bit i
    for (uint32_t d : {1u, 2u, 3u, 7u, 20u, 100u, 1000u, 1500u, 4096u, 10000u, 65537u, 1000003u, 2147483647u}) {
        const unsigned long long m = magic64(d);
        const uint32_t edge[] = {0u, 1u, d - 1u, d, d + 1u, 0xFFFFFFFFu, 0x80000000u, 2u * d - 1u};
        for (uint32_t i : edge) CHECK(div_magic64(i, m) == i / d, "div_magic64(%u, d %u)", i, d);
        for (int n = 0; n < 200000; ++n) {
            const uint32_t i = next32();
            if (div_magic64(i, m) != i / d) { CHECK(false, "div_magic64(%u, d %u)", i, d); break; }
        }
    }
    // cos(2 pi v): exact at the integers and half-integers, within 2.5e-7 everywhere
    double worst = 0.0;
    for (int n = 0; n < 4000000; ++n) {
        const float v = -600.f + 1200.f * (float)n / 4000000.f;
        const double e = std::fabs((double)cos2pi(v) - std::cos(2.0 * M_PI * (double)v));
        if (e > worst) worst = e;
    }
    for (int n = 0; n < 1000000; ++n) {   // fine grid on [-1, 1]
        const float v = -1.f + 2.f * (float)n / 1000000.f;
        const double e = std::fabs((double)cos2pi(v) - std::cos(2.0 * M_PI * (double)v));
        if (e > worst) worst = e;
    }
    CHECK(worst <= 2.5e-7, "cos2pi worst error %.3e", worst);
    for (int k = -300; k <= 300; ++k) {
        CHECK(cos2pi((float)k) == 1.f, "cos2pi(%d)", k);
        CHECK(cos2pi((float)k + 0.5f) == -1.f, "cos2pi(%d + 1/2)", k);
    }
    // the terms: zero at their optima, close to the double-precision formulas
    CHECK(rast_term(0.f) == 0.f, "rast_term(0)");
    CHECK(rosen_term(1.f, 1.f) == 0.f, "rosen_term(1, 1)");
    double wr = 0.0, wq = 0.0;
    for (int n = 0; n < 200000; ++n) {
        const float v = ((float)(next32() >> 8) / 16777216.f - 0.5f) * 200.f;
        const float w = ((float)(next32() >> 8) / 16777216.f - 0.5f) * 200.f;
        const double a = (double)w - (double)v * v, b = (double)v - 1.0;
        const double rd = 100.0 * a * a + b * b;
        const double qd = (double)v * v - 10.0 * std::cos(2.0 * M_PI * (double)v) + 10.0;
        wr = std::fmax(wr, std::fabs(rosen_term(v, w) - rd) / std::fmax(1.0, rd));
        wq = std::fmax(wq, std::fabs(rast_term(v) - qd) / std::fmax(1.0, qd));
    }
    CHECK(wr <= 1e-6, "rosen_term worst relative error %.3e", wr);
    CHECK(wq <= 1e-6, "rast_term worst relative error %.3e", wq);
    std::printf("cos2pi %.3e rosen %.3e rast %.3e fails %d\n", worst, wr, wq, fails);
    return fails == 0 ? 0 : 1;
}
"""


def test_division_cosine_and_terms_on_the_host(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "arith_check.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "arith_check"
    cmd = [nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-Xcompiler",
           "-ffp-contract=off", "-I", os.path.join(ROOT, "include"), "-I", CSRC, str(src), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
