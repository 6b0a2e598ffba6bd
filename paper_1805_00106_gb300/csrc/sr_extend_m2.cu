// sr_extend_m2.cu -- instantiations of the int16 extension kernel for readout mode 2
// (end-row search of winning windows).
#include "sr_extend.cuh"

namespace sr {

int dispatch_mode2(uint32_t lanes, uint32_t rows, const ExtArgs& a, cudaStream_t st) {
#define SR_CASE(g, r) \
  if (lanes == g && rows == r) return launch16<g, r, 2, true>(a, st, 0);
  SR_SHAPES(SR_CASE)
#undef SR_CASE
  return -1;
}

int preload_mode2() {
  int n_ = 0;
#define SR_CASE(g, r) SR_TOUCH((k_extend16<g, r, 2, true>));
  SR_SHAPES(SR_CASE)
#undef SR_CASE
  return n_;
}

}  // namespace sr
