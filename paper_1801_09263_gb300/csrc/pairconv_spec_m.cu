// Size-specialised FP32 pair-convolution passes for n in {60, 64, 72, 80}.
#include "pairconv_spec2.cuh"

namespace lace {

bool spec_launch_m(int pass, int n, int nb, const ConvArgs<float>& P, int g0, cudaStream_t s) {
    switch (n) {
        case 60: return spec::launch_any<60>(pass, nb, P, g0, s);
        case 64: return spec::launch_any<64>(pass, nb, P, g0, s);
        case 72: return spec::launch_any<72>(pass, nb, P, g0, s);
        case 80: return spec::launch_any<80>(pass, nb, P, g0, s);
        default: return false;
    }
}

}  // namespace lace
