"""Host-side planning rules of libtdse (tdse_internal.h), compiled with the host compiler and
checked over their whole input range (no GPU): the halo length makes the truncated sweeps exact to
double rounding (beta^K < 1e-18), segment counts stay within the CTA and leave every segment at
least four halos long, and the segment length of a group covers its grid."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2507_04115_gb300", "csrc")

PROGRAM = r"""
#include <cmath>
#include <cstdio>
#include "tdse_internal.h"
using namespace tdse;
int main() {
    int bad = 0;
    for (int i = 0; i <= 100000; ++i) {
        const double beta = 0.9 * i / 100000.0;
        const int K = halo_for_beta(beta);
        if (beta >= 0.85) { if (K != 0) { std::printf("beta %g: K %d, want 0\n", beta, K); ++bad; } continue; }
        if (K < 8) { std::printf("beta %g: K %d < 8\n", beta, K); ++bad; }
        if (beta >= 1e-3 && !(std::pow(beta, K) < 1e-18)) { std::printf("beta %g: beta^K = %g\n", beta, std::pow(beta, K)); ++bad; }
        if (K > 8 && std::pow(beta, K - 1) < 1e-18) { std::printf("beta %g: K %d not minimal\n", beta, K); ++bad; }
    }
    for (int N = 16; N <= 20000; N += 7)
        for (int K = 0; K <= 300; K += 13)
            for (int w = 1; w <= kMaxSegments; ++w) {
                const int P = class_segments(N, K, w);
                if (P < 1 || P > w) { std::printf("N %d K %d w %d: P %d\n", N, K, w, P); ++bad; }
                if (K == 0 && P != 1) { std::printf("N %d: no halo but P %d\n", N, P); ++bad; }
                if (P > 1 && N / P < 4 * K) { std::printf("N %d K %d: segment %d < 4K\n", N, K, N / P); ++bad; }
                for (int L = 1; L <= 32; L *= 2) {
                    const int m = group_segment_length(N, P, L);
                    if ((long)m * P * L < N || (long)(m - 1) * P * L >= N) {
                        std::printf("N %d P %d L %d: m %d\n", N, P, L, m); ++bad;
                    }
                }
            }
    std::printf("%d violations\n", bad);
    return bad ? 1 : 0;
}
"""


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def test_planning_rules(tmp_path):
    inc = _cuda_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "rules.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "rules"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", inc,
                           str(src), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:]


RING_PROGRAM = r"""
#include <cstdio>
#include "tdse_sched.cuh"
using namespace tdse;
int main() {
    int bad = 0;
    for (int P = 1; P <= kMaxSegments; ++P)
        for (int per_sm = 1; per_sm <= 4; ++per_sm) {
            const int r = full_cn_ring_slots(P, per_sm);
            if (r < kMinRing || r > kMaxRing) { std::printf("P %d per_sm %d: ring %d\n", P, per_sm, r); ++bad; }
            // more slots only when they fit: per_sm CTAs of this size share 220 KB
            if (r > kMinRing && (size_t)per_sm * full_cn_smem_bytes(1, P, r) > 220u * 1024u) {
                std::printf("P %d per_sm %d: %zu bytes x %d\n", P, per_sm, full_cn_smem_bytes(1, P, r), per_sm); ++bad;
            }
            if (r < kMaxRing && (size_t)per_sm * full_cn_smem_bytes(1, P, r + 1) <= 220u * 1024u) {
                std::printf("P %d per_sm %d: ring %d could be deeper\n", P, per_sm, r); ++bad;
            }
        }
    // one CTA of any width fits the 227 KB a CTA may use
    if (full_cn_smem_max_bytes() > 227u * 1024u) { std::printf("max %zu\n", full_cn_smem_max_bytes()); ++bad; }
    std::printf("%d violations\n", bad);
    return bad ? 1 : 0;
}
"""


def test_mixed_ring_depth_fits_shared_memory(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("needs nvcc")
    src = tmp_path / "ring.cu"
    src.write_text(RING_PROGRAM)
    exe = tmp_path / "ring"
    subprocess.check_call([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:]


WIDTH_PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include "tdse_internal.h"
using namespace tdse;
static int bad = 0;
#define CHECK(c, ...) do { if (!(c)) { std::printf(__VA_ARGS__); std::printf("\n"); ++bad; } } while (0)

// groups cover every instance of every class, widths are powers of two >= the base
static void check_cover(const std::vector<WidthClass>& cls, const std::vector<std::vector<int>>& w)
{
    for (size_t c = 0; c < cls.size(); ++c) {
        int64_t covered = 0;
        for (int L : w[c]) {
            CHECK(L >= cls[c].L_base && L <= 32 && (L & (L - 1)) == 0, "class %zu: width %d", c, L);
            CHECK(cls[c].K > 0 || L == 1, "class %zu without halo split to %d", c, L);
            covered += 32 / L;
        }
        const int64_t n = (int64_t)cls[c].nt_desc.size();
        CHECK(covered >= n, "class %zu: %lld of %lld covered", c, (long long)covered, (long long)n);
        CHECK(w[c].empty() || covered - 32 / w[c].back() < n, "class %zu: an empty group", c);
    }
}

int main() {
    const double inf = std::numeric_limits<double>::infinity();
    std::vector<std::vector<int>> w, w0;
    // equal pulses, enough groups to fill the SMs (the 8192 x 4096 volume): nothing is split
    {
        std::vector<WidthClass> v{{4096, 28, 1, std::vector<int64_t>(8192, 55159)}};
        const double M = plan_widths(v, 8, 152, &w);
        const double M0 = plan_widths_at(v, 8, 152, inf, &w0);
        check_cover(v, w);
        CHECK(w == w0 && M == M0, "volume batch split");
        for (int L : w[0]) CHECK(L == 1, "volume width %d", L);
    }
    // equal pulses on few groups (1024 x 2048 at base L = 4): splitting further cannot help
    {
        std::vector<WidthClass> v{{2048, 28, 4, std::vector<int64_t>(1024, 33095)}};
        plan_widths(v, 8, 152, &w);
        check_cover(v, w);
        for (int L : w[0]) CHECK(L == 4, "adjoint batch width %d", L);
    }
    // one instance at base L = 32 stays there; a class without halo stays at 1
    {
        std::vector<WidthClass> v{{2000, 36, 32, {8818}}, {64, 0, 1, {100, 90}}};
        plan_widths(v, 8, 152, &w);
        check_cover(v, w);
        CHECK(w[0].size() == 1 && w[0][0] == 32, "single atom");
        CHECK(w[1].size() == 1 && w[1][0] == 1, "no-halo class");
    }
    // uneven pulses on uneven grids (LCG-drawn, as the 16384-instance uneven batch): the longest
    // groups are widened, the estimate improves by at least 5 %, and no group is longer than the
    // work per SM afterwards
    {
        const int Ns[4] = {1024, 2048, 4096, 8192};
        const int Ks[2] = {28, 20};
        std::vector<WidthClass> v;
        for (int a = 0; a < 4; ++a)
            for (int k = 0; k < 2; ++k) v.push_back({Ns[a], Ks[k], 1, {}});
        uint64_t s = 12345;
        for (int i = 0; i < 16384; ++i) {
            s = s * 6364136223846793005ull + 1442695040888963407ull;
            const int c = (int)((s >> 33) % 8);
            const int64_t nt = 8800 + (int64_t)((s >> 13) % 190000);
            v[c].nt_desc.push_back(nt);
        }
        for (auto& C : v) std::sort(C.nt_desc.begin(), C.nt_desc.end(), std::greater<int64_t>());
        const double M0 = plan_widths_at(v, 8, 152, inf, &w0);
        const double M = plan_widths(v, 8, 152, &w);
        check_cover(v, w);
        CHECK(M < 0.95 * M0, "uneven: estimate %g vs %g", M, M0);
        int split = 0;
        double work = 0.0, longest = 0.0;
        for (size_t c = 0; c < v.size(); ++c) {
            int64_t k = 0;
            for (int L : w[c]) {
                const double t = (double)v[c].nt_desc[k] * group_step_cost(v[c].N, v[c].K, L, 8);
                work += t;
                longest = std::max(longest, t);
                split += L > 1;
                k += 32 / L;
            }
        }
        CHECK(split > 0, "uneven: nothing split");
        CHECK(longest <= work / 152 * 1.0001, "uneven: longest group %g above work per SM %g", longest, work / 152);
        CHECK(std::fabs(std::max(work / 152, longest) - M) <= 1e-9 * M, "uneven: estimate mismatch");
    }
    std::printf("%d violations\n", bad);
    return bad ? 1 : 0;
}
"""


def test_group_widths_by_makespan(tmp_path):
    """The planner's group widths (plan_widths): equal-length batches keep the per-step model's
    width, an uneven batch gets its longest groups spread over more lanes so that no group outlasts
    the work per SM, and the groups always cover every instance."""
    inc = _cuda_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "widths.cpp"
    src.write_text(WIDTH_PROGRAM)
    exe = tmp_path / "widths"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", inc,
                           str(src), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:]
