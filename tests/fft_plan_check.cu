// Host-only checks of the launch plans of the out-of-place FFT passes
// (pairconv_spec2.cuh) for every size-specialised cubic grid: a two-radix
// plan, thread counts, register caps and shared memory that fit one SM at
// the planned number of CTAs, and the alignment of their 16-byte accesses
// (orbital and W planes, the K(G)/Ng slab rows, the plane buffers in shared
// memory).  Prints one line per size; exit code = number of failed checks.
#include <cstdio>

#include "pairconv_spec2.cuh"

int main() {
    using namespace lace::spec2;
    const int sizes[] = {24, 32, 36, 40, 48, 50, 54, 60, 64, 72, 80, 96, 100};
    int bad = 0;
    for (int n : sizes) {
        const Plan2 p = plan2(n);
        const int nt = threads_for(n), m = blocks_at(n, nt), regs = max_regs(n);
        const int warps = (nt + 31) / 32;
        const int a = n * (n / p.r1), b = n * (n / p.r2);  // butterflies of the two stage kinds
        const int lo = ((a < b ? a : b) + 31) / 32 * 32;
        int fails = 0;
        if (p.r1 * p.r2 != n || !lace::spec::radix_ok(p.r1) || !lace::spec::radix_ok(p.r2)) ++fails;
        if (nt % 32 || nt > 1024 || nt < (lo < 1024 ? lo : 1024)) ++fails;
        if (m < 1 || m * nt > 2048) ++fails;
        if (regs < 40 || regs > 255 || regs % 8) ++fails;
        // registers: every warp draws on one of four 16K sub-partition files
        if ((m * warps + 3) / 4 * 32 * regs > 16384) ++fails;
        // shared memory: m CTAs of the largest pass plus 1 KB reserved each
        if ((size_t)m * (smem_max(n) + 1024) > 227u * 1024u) ++fails;
        for (int pass = 0; pass < 3; ++pass)
            if (smem_bytes(n, pass) + 1024 > 227u * 1024u) ++fails;
        // 16-byte accesses: a plane of n^2 FP32 values and a grid of n^3 start
        // on 16-byte boundaries (pass A's rho loads, pass C's W reductions);
        // the second plane buffer (after n (n + 1) complex values) too; the
        // K(G)/Ng slab is copied in 16-byte pieces of table rows of n floats
        if ((n * n * 4) % 16 || ((size_t)n * n * n * 4) % 16 || (n * (n + 1) * 8) % 16) ++fails;
        if (kslab_fits(n) && (n * 4) % 16) ++fails;
        std::printf("n=%d plan=%dx%d threads=%d ctas=%d regs=%d smem_max=%zu kslab=%d %s\n", n, p.r1, p.r2, nt, m,
                    regs, smem_max(n), (int)kslab_fits(n), fails ? "FAIL" : "ok");
        bad += fails;
    }
    return bad;
}
