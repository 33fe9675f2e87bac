// Size-specialised FP32 pair-convolution passes for n in {24, 32, 36, 40, 48}.
#include "pairconv_spec2.cuh"

namespace lace {

bool spec_launch_s(int pass, int n, int nb, const ConvArgs<float>& P, int g0, cudaStream_t s) {
    switch (n) {
        case 24: return spec::launch_any<24>(pass, nb, P, g0, s);
        case 32: return spec::launch_any<32>(pass, nb, P, g0, s);
        case 36: return spec::launch_any<36>(pass, nb, P, g0, s);
        case 40: return spec::launch_any<40>(pass, nb, P, g0, s);
        case 48: return spec::launch_any<48>(pass, nb, P, g0, s);
        default: return false;
    }
}

// Sizes whose one-grid out-of-place passes exist (they take merged launches).
bool spec_merge_ok(int n) {
    switch (n) {
        case 24: return spec2::smem_max(24) <= 200 * 1024;
        case 32: return spec2::smem_max(32) <= 200 * 1024;
        case 36: return spec2::smem_max(36) <= 200 * 1024;
        case 40: return spec2::smem_max(40) <= 200 * 1024;
        case 48: return spec2::smem_max(48) <= 200 * 1024;
        case 50: return spec2::smem_max(50) <= 200 * 1024;
        case 54: return spec2::smem_max(54) <= 200 * 1024;
        case 60: return spec2::smem_max(60) <= 200 * 1024;
        case 64: return spec2::smem_max(64) <= 200 * 1024;
        case 72: return spec2::smem_max(72) <= 200 * 1024;
        case 80: return spec2::smem_max(80) <= 200 * 1024;
        case 96: return spec2::smem_max(96) <= 200 * 1024;
        case 100: return spec2::smem_max(100) <= 200 * 1024;
        case 128: return spec2::smem_max(128) <= 200 * 1024;
        default: return false;
    }
}

}  // namespace lace
