// Batched filter, one pair per lane, tiles of 9..12 words per read.
#include "batched.cuh"

namespace gk {

cudaError_t launch_whole_w9_12(const BatchArgs &a, uint32_t sms, uint32_t bpsm, uint32_t wpb, cudaStream_t s) {
  return launch_whole<9, 12, 2>(a, sms, bpsm, wpb, s);
}

}  // namespace gk
