"""The radix orders of the line FFT (host side, no GPU): for every side
n = 2^5 .. 2^12 and order, the runtime sequence (setup_kernels.cuh) and the
compile-time one (Seq in fft_core.cuh) agree with the sequence restated here
(radix-16 passes, and the one radix-2/4/8 pass last, first or second), the
radices multiply to n, and the pass-major twiddle table holds
sum over passes p >= 1 of (R_p - 1) Ns_p = n - R_0 entries."""
import os
import shutil
import subprocess
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1410_2855_gb300", "csrc")


def expected(logn, order):
    p16, small = logn // 4, logn % 4
    seq = [16] * p16
    if small:
        pos = len(seq) if order == 0 else (0 if order == 1 or p16 < 2 else 1)
        seq.insert(pos, 1 << small)
    return seq


def orders(logn):
    return 1 if logn % 4 == 0 else (3 if logn // 4 >= 2 else 2)


def test_sequences_spans_and_table_sizes(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "seq.cu"
    src.write_text(textwrap.dedent("""
        #include <cstdio>
        #include "fft_core.cuh"
        #include "setup_kernels.cuh"
        using namespace rtk;
        template <int L, int O> void row() {
            using S = Seq<L, O>;
            std::printf("%d %d %d %d", L, O, S::NP, S::tw_size());
            for (int p = 0; p < S::NP; ++p) std::printf(" %d/%d", S::radix(p), S::span(p));
            std::printf(" | %d %d", seq_passes(L), twiddle_count(L, O));
            for (int p = 0; p < seq_passes(L); ++p) std::printf(" %d", seq_radix(L, O, p));
            std::printf(" | %d\\n", radix_orders(L));
        }
        template <int L> void rows() {
            row<L, 0>();
            if constexpr (radix_orders(L) > 1) row<L, 1>();
            if constexpr (radix_orders(L) > 2) row<L, 2>();
        }
        int main() { rows<5>(); rows<6>(); rows<7>(); rows<8>(); rows<9>(); rows<10>(); rows<11>(); rows<12>(); }
    """))
    exe = tmp_path / "seq"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "--expt-relaxed-constexpr",
                    "-I", CSRC, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    seen = set()
    for line in filter(None, out):
        head, runtime, norders = line.split(" | ")
        f = head.split()
        logn, order, npass, tw = int(f[0]), int(f[1]), int(f[2]), int(f[3])
        pairs = [tuple(map(int, x.split("/"))) for x in f[4:]]
        want = expected(logn, order)
        assert [r for r, _ in pairs] == want and npass == len(want)
        span = 1
        for r, ns in pairs:
            assert ns == span
            span *= r
        assert span == 1 << logn
        assert tw == sum((r - 1) * ns for r, ns in pairs[1:]) == (1 << logn) - want[0]
        rt = runtime.split()
        assert int(rt[0]) == npass and int(rt[1]) == tw and list(map(int, rt[2:])) == want
        assert int(norders) == orders(logn)
        seen.add((logn, order))
    assert seen == {(L, o) for L in range(5, 13) for o in range(orders(L))}
