// The persistent multi-instance kernel at 512 threads a CTA and two CTAs an
// SM (64 registers a thread), with the size-specialised pass bodies in
// thread groups (a translation unit of its own so that the build compiles it
// in parallel with the others).
#include "pairconv_multi.cuh"

namespace lace {

const void* multi_kernel_512x2() { return (const void*)multi::pairconv_multi_kernel<512, true, 2>; }

}  // namespace lace
