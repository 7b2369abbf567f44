// Mixed-precision Chebyshev filter on tcgen05 tensor cores (BF16 x3 split products).
#include "solver.cuh"

namespace cb {

bool mixed_available() { return false; }

int filter_mixed_sorted(const cplx*, const cplx*, int64_t, cplx*, int64_t, const int*, double, double, double, cplx*,
                        cudaStream_t, FilterStats*) {
  return CHASE_BSE_UNSUPPORTED;
}

}  // namespace cb
