"""Host-side checks of the shared-memory layout of the cooperative grid kernel
(csrc/apo_plan.h) and of the canonical operand layout of its tcgen05 rotation
(umma_off in csrc/apo_device.cuh).  A small C++ program includes the headers,
is compiled with nvcc and runs on the host only (no GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_14982_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "apo_plan.h"
using namespace apo;

static int fails = 0;
#define CHECK(c, ...) do { if (!(c)) { ++fails; std::printf("FAIL " __VA_ARGS__); std::printf("\n"); } } while (0)

static apo_problem make(int D, int ncomp, bool rotated, bool canonical)
{
    apo_problem P{};
    const int Dp = (D + 3) & ~3, Np = (D + 15) & ~15;
    P.D = D; P.Dp = Dp; P.Np = Np; P.ncomp = ncomp; P.any_rot = rotated ? 1 : 0; P.kind = ncomp > 1 ? 7 : 3;
    P.dev.D = D; P.dev.Dp = Dp; P.dev.Np = Np; P.dev.ncomp = ncomp; P.dev.bws = split_words(D);
    for (int c = 0; c < ncomp; ++c) P.dev.comp[c].MT = rotated ? (const float*)16 : nullptr;
    P.dev.comp[0].Th = canonical ? (const uint4*)16 : nullptr;
    return P;
}

int main()
{
    const size_t smem_max = 232448 - 2048;
    int tc_plans = 0;
    for (int D : {1, 3, 10, 16, 37, 50, 64, 100, 112, 126, 128}) {
        for (int ps : {128, 300, 1500, 4096, 8192}) {
            apo_problem P = make(D, 1, true, D <= kTcM);
            const SmemPlan L = choose_plan(&P, ps, false, true, smem_max);
            const int Np = P.Np;
            CHECK(L.total <= smem_max, "D %d ps %d: plan of %u bytes", D, ps, L.total);
            if (!L.tc) continue;
            ++tc_plans;
            const size_t ta_end = (size_t)L.TA + 4u * Np * Np, ty_end = (size_t)L.TY + 4u * kTcN * Np;
            CHECK(L.TA % 16 == 0 && L.TY % 16 == 0, "D %d ps %d: TA/TY alignment", D, ps);
            CHECK(L.chunk == kTcN && !L.mt_smem, "D %d ps %d: chunk %d, mt_smem %d", D, ps, L.chunk, L.mt_smem);
            // the lo part's MMAs read kTcM rows: the rows past Np must stay inside TY
            CHECK(L.TY == ta_end, "D %d ps %d: TY not directly after TA", D, ps);
            CHECK((size_t)L.TA + 2u * Np * Np + 2u * kTcM * Np <= ty_end, "D %d ps %d: over-read past TY", D, ps);
            CHECK(ty_end <= L.o && ty_end <= L.total, "D %d ps %d: TY overlaps the next region", D, ps);
            // the regions carved before TA end at or before it
            for (uint32_t off : {L.perm0, L.perm1, L.keys, L.MT}) CHECK(off <= L.TA, "D %d ps %d: region order", D, ps);
        }
        // never for compositions, unrotated objectives or D > kTcM
        apo_problem C = make(D, 3, true, false);
        CHECK(!choose_plan(&C, 4096, false, true, smem_max).tc, "D %d: composition got a tcgen05 plan", D);
        apo_problem U = make(D, 1, false, false);
        CHECK(!choose_plan(&U, 4096, false, true, smem_max).tc, "D %d: unrotated objective got a tcgen05 plan", D);
        apo_problem Q = make(D, 1, true, D <= kTcM);
        CHECK(!choose_plan(&Q, 300, true, false, smem_max).tc, "D %d: work-queue plan got tcgen05", D);
    }
    apo_problem B = make(200, 1, true, false);
    CHECK(!choose_plan(&B, 4096, false, true, smem_max).tc, "D 200 got a tcgen05 plan");

    // work-queue plans: 64-row chunks when they fit the budget, else 32-row
    // ones; a preferred chunk is honoured; nothing that fits with 32-row
    // chunks is refused
    int q64 = 0, q32 = 0;
    for (int D : {10, 20, 50, 100, 200}) {
        for (int ps : {20, 77, 300, 512, 1024}) {
            for (size_t budget : {(size_t)56 * 1024, (size_t)75 * 1024, (size_t)113 * 1024, smem_max}) {
                for (bool res : {true, false}) {
                    apo_problem P = make(D, 1, true, false);
                    const SmemPlan L = choose_plan(&P, ps, res, false, budget);
                    const SmemPlan S32 = make_smem_plan(&P, ps, res, false, false, kChunk);
                    if (L.total <= budget) {
                        CHECK(L.chunk == kQueueChunk || L.chunk == kChunk, "D %d ps %d: chunk %d", D, ps, L.chunk);
                        if (L.chunk == kChunk)
                            CHECK(make_smem_plan(&P, ps, res, false, false, kQueueChunk).total > budget,
                                  "D %d ps %d: 32-row chunks although 64 fit", D, ps);
                        q64 += L.chunk == kQueueChunk;
                        q32 += L.chunk == kChunk;
                    } else {
                        CHECK(S32.total > budget, "D %d ps %d res %d: refused although 32-row chunks fit", D, ps, (int)res);
                    }
                    const SmemPlan Lp = choose_plan(&P, ps, res, false, budget, kChunk);
                    if (Lp.total <= budget) CHECK(Lp.chunk == kChunk, "D %d ps %d: preferred chunk ignored", D, ps);
                }
            }
        }
    }
    CHECK(q64 > 0 && q32 > 0, "work-queue plans: %d with 64-row and %d with 32-row chunks", q64, q32);

    // canonical K-major layout: a bijection onto the operand's bytes, 8-row x
    // 16-byte core matrices, K-adjacent ones 128 bytes apart (the descriptor's
    // leading offset), 8-row groups Kt * 16 bytes apart (its stride offset)
    for (int R : {8, 64, 128}) {
        for (int Kt : {16, 48, 112, 128}) {
            std::vector<int> seen((size_t)R * Kt, 0);
            for (int r = 0; r < R; ++r)
                for (int k = 0; k < Kt; ++k) {
                    const uint32_t o = umma_off(r, k, Kt);
                    CHECK(o % 2 == 0 && o < 2u * R * Kt, "umma_off(%d, %d, %d) = %u out of range", r, k, Kt, o);
                    if (o % 2 == 0 && o < 2u * R * Kt) seen[o / 2] += 1;
                    CHECK(umma_off(r, k, Kt) - umma_off(r & ~7, k & ~7, Kt) == (uint32_t)(16 * (r & 7) + 2 * (k & 7)),
                          "core matrix of (%d, %d)", r, k);
                    if (k >= 8) CHECK(umma_off(r, k, Kt) - umma_off(r, k - 8, Kt) == 128u, "LBO at (%d, %d)", r, k);
                    if (r >= 8) CHECK(umma_off(r, k, Kt) - umma_off(r - 8, k, Kt) == 16u * Kt, "SBO at (%d, %d)", r, k);
                }
            for (int v : seen) CHECK(v == 1, "umma_off not a bijection (R %d, Kt %d)", R, Kt);
        }
    }
    std::printf("tc_plans %d fails %d\n", tc_plans, fails);
    return fails != 0;
}
"""


def test_grid_plan_and_operand_layout(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "plan_check.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "plan_check"
    cmd = [nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", os.path.join(ROOT, "include"),
           "-I", CSRC, str(src), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    # layouts up to D 112 at ps 4096 (and the smaller ones) take tcgen05
    tc_plans = int(out.stdout.split("tc_plans")[1].split()[0])
    assert tc_plans >= 40, out.stdout
