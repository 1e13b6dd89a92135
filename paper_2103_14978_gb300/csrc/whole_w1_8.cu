// Batched filter, one pair per lane, tiles of 1..8 words per read.
#include "batched.cuh"

namespace gk {

cudaError_t launch_whole_w1_8(const BatchArgs &a, uint32_t sms, uint32_t bpsm, uint32_t wpb, cudaStream_t s) {
  return launch_whole<1, 8, 0>(a, sms, bpsm, wpb, s);
}

}  // namespace gk
