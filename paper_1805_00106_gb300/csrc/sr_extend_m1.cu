// sr_extend_m1.cu -- instantiations of the int16 extension kernel for readout mode 1
// (best cell of the final row).
#include "sr_extend.cuh"

namespace sr {

int dispatch_mode1(bool persist, uint32_t lanes, uint32_t rows, const ExtArgs& a, cudaStream_t st,
                   uint64_t plain_tasks) {
  if (!persist) {
#define SR_CASE(g, r) \
  if (lanes == g && rows == r) return launch16<g, r, 1, false>(a, st, plain_tasks);
    SR_PLAIN_SHAPES(SR_CASE)
#undef SR_CASE
    return -1;
  }
#define SR_CASE(g, r) \
  if (lanes == g && rows == r) return launch16<g, r, 1, true>(a, st, 0);
  SR_SHAPES(SR_CASE)
#undef SR_CASE
  return -1;
}

int preload_mode1() {
  int n_ = 0;
#define SR_CASE(g, r) SR_TOUCH((k_extend16<g, r, 1, true>));
  SR_SHAPES(SR_CASE)
#undef SR_CASE
#define SR_CASE(g, r) SR_TOUCH((k_extend16<g, r, 1, false>));
  SR_PLAIN_SHAPES(SR_CASE)
#undef SR_CASE
  return n_;
}

}  // namespace sr
