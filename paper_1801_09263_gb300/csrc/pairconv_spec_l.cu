// Size-specialised FP32 pair-convolution passes for n in {96, 100, 128}.
#include "pairconv_spec2.cuh"

namespace lace {

bool spec_launch_l(int pass, int n, int nb, const ConvArgs<float>& P, int g0, cudaStream_t s) {
    switch (n) {
        case 96: return spec::launch_any<96>(pass, nb, P, g0, s);
        case 100: return spec::launch_any<100>(pass, nb, P, g0, s);
        case 128: return spec::launch_any<128>(pass, nb, P, g0, s);
        default: return false;
    }
}

}  // namespace lace
