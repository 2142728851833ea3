"""The serving engine's request pool (csrc/pool.h) on the host: a seeded
random sequence of allocations and releases is checked, step by step, against
a brute-force model of first-fit over the gaps between live blocks.

Checked: every block starts on a 256-byte boundary, lies inside the range and
overlaps no live block; an allocation succeeds exactly when some gap holds it
and then returns the lowest such gap (first fit over fully coalesced free
space); bytes in use and the peak are the sums of the live blocks' aligned
sizes; once everything is released, one block of the whole range fits again.
The pool makes no CUDA call, so g++ builds the check without a GPU.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1705_10087_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <vector>
#include <algorithm>
#include "pool.h"

using csc::Pool;
using csc::align_up;
using csc::kAlign;

static uint64_t st = 0x9E3779B97F4A7C15ull;
static uint64_t rnd() { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return st; }

#define CHECK(c, ...) do { if (!(c)) { std::printf("FAIL line %d: ", __LINE__); \
    std::printf(__VA_ARGS__); std::printf("\n"); return 1; } } while (0)

struct Blk { size_t off, len; };

// first gap (lowest offset) between live blocks that holds n bytes
static bool model_fit(const std::vector<Blk> &live, size_t size, size_t n, size_t *off)
{
    std::vector<Blk> s(live);
    std::sort(s.begin(), s.end(), [](const Blk &a, const Blk &b) { return a.off < b.off; });
    size_t cur = 0;
    for (const Blk &b : s) {
        if (b.off - cur >= n) { *off = cur; return true; }
        cur = b.off + b.len;
    }
    if (size - cur >= n) { *off = cur; return true; }
    return false;
}

int main(int argc, char **argv)
{
    const size_t size = (size_t)std::strtoull(argv[1], nullptr, 10);
    const int steps = std::atoi(argv[2]);
    st ^= (uint64_t)std::strtoull(argv[3], nullptr, 10) * 0x2545F4914F6CDD1Dull;
    Pool p;
    p.init(nullptr, size);
    std::vector<Blk> live;
    size_t used = 0, peak = 0;
    int allocs = 0, fails = 0;
    for (int i = 0; i < steps; i++) {
        const bool do_alloc = live.empty() || rnd() % 100 < 55;
        if (do_alloc) {
            // sizes from 1 byte to a quarter of the range, many not multiples of 256
            size_t n = 1 + rnd() % (size / 4);
            if (rnd() % 4 == 0) n = (1 + rnd() % 8) * kAlign;
            size_t want = 0, got = 0;
            const bool fits = model_fit(live, size, align_up(n), &want);
            const bool ok = p.alloc(n, &got);
            CHECK(ok == fits, "step %d: alloc(%zu) ok=%d model=%d", i, n, (int)ok, (int)fits);
            if (!ok) { fails++; continue; }
            CHECK(got == want, "step %d: first fit at %zu, model %zu", i, got, want);
            CHECK(got % kAlign == 0, "step %d: offset %zu unaligned", i, got);
            CHECK(got + align_up(n) <= size, "step %d: block past the range", i);
            for (const Blk &b : live)
                CHECK(got + align_up(n) <= b.off || b.off + b.len <= got,
                      "step %d: overlap with [%zu,+%zu)", i, b.off, b.len);
            live.push_back({got, align_up(n)});
            used += align_up(n);
            peak = std::max(peak, used);
            allocs++;
        } else {
            const size_t j = rnd() % live.size();
            p.release(live[j].off, live[j].len - (rnd() % 2 ? 0 : (rnd() % kAlign)));
            used -= live[j].len;
            live.erase(live.begin() + (long)j);
        }
        CHECK(p.in_use == used, "step %d: in_use %zu, model %zu", i, p.in_use, used);
        CHECK(p.peak == peak, "step %d: peak %zu, model %zu", i, p.peak, peak);
    }
    for (const Blk &b : live)
        p.release(b.off, b.len);
    CHECK(p.in_use == 0, "in_use %zu after releasing everything", p.in_use);
    size_t off = 1;
    CHECK(p.alloc(size, &off) && off == 0, "whole range does not fit after full release");
    std::printf("ok %d %d\n", allocs, fails);
    return 0;
}
"""


@pytest.mark.parametrize("size,steps,seed", [(1 << 20, 4000, 1), (1 << 20, 4000, 2),
                                             (40 * 256 + 77 * 256, 3000, 3)])
def test_pool_first_fit_against_model(tmp_path, size, steps, seed):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "pool_check.cc"
    src.write_text(DRIVER)
    exe = tmp_path / "pool_check"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", CSRC, "-o", str(exe), str(src)])
    res = subprocess.run([str(exe), str(size), str(steps), str(seed)], capture_output=True,
                         text=True, timeout=120)
    assert res.returncode == 0, res.stdout + res.stderr
    tag, allocs, fails = res.stdout.split()
    assert tag == "ok" and int(allocs) > steps // 4 and int(fails) > 0
