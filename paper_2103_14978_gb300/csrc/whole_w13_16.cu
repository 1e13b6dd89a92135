// Batched filter, one pair per lane, tiles of 13..16 words per read.
#include "batched.cuh"

namespace gk {

cudaError_t launch_whole_w13_16(const BatchArgs &a, uint32_t sms, uint32_t bpsm, uint32_t wpb, cudaStream_t s) {
  return launch_whole<13, 16, 3>(a, sms, bpsm, wpb, s);
}

}  // namespace gk
