// Size-specialised FP32 pair-convolution passes for n in {24, 32, 36, 40, 48}.
#include "pairconv_pair.cuh"

namespace lace {

bool spec_launch_s(int pass, int n, int nb, const ConvArgs<float>& P, int g0, cudaStream_t s, bool allow_pair) {
    switch (n) {
        case 24: return spec::launch_any<24>(pass, nb, P, g0, s, allow_pair);
        case 32: return spec::launch_any<32>(pass, nb, P, g0, s, allow_pair);
        case 36: return spec::launch_any<36>(pass, nb, P, g0, s, allow_pair);
        case 40: return spec::launch_any<40>(pass, nb, P, g0, s, allow_pair);
        case 48: return spec::launch_any<48>(pass, nb, P, g0, s, allow_pair);
        default: return false;
    }
}

}  // namespace lace
