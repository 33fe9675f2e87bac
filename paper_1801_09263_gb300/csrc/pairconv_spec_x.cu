// Size-specialised FP32 pair-convolution passes for n in {50, 54}.
#include "pairconv_spec2.cuh"

namespace lace {

bool spec_launch_x(int pass, int n, int nb, const ConvArgs<float>& P, int g0, cudaStream_t s) {
    switch (n) {
        case 50: return spec::launch_any<50>(pass, nb, P, g0, s);
        case 54: return spec::launch_any<54>(pass, nb, P, g0, s);
        default: return false;
    }
}

}  // namespace lace
