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
