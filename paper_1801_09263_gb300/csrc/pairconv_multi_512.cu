// The persistent multi-instance kernel at 512 threads a CTA, with the
// size-specialised pass bodies (a translation unit of its own so that the
// build compiles it in parallel with the others).
#include "pairconv_multi.cuh"

namespace lace {

const void* multi_kernel_512() { return (const void*)multi::pairconv_multi_kernel<512, true>; }

}  // namespace lace
