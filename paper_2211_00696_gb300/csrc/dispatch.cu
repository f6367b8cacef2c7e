// Precision dispatch for the apply path.
#include "plan.h"

namespace phikron {

int apply_dispatch(Plan& P, int nrhs, const double* V, double* Out, cudaStream_t st) {
  const long long N = P.N;
  for (int r = 0; r < nrhs; ++r) {
    if (P.opts.precision == PHIKRON_PREC_OZAKI_BF16)
      PK_RET(apply_mixed(P, V + (size_t)r * N, Out + (size_t)r * (P.p + 1) * (P.opts.half_step ? 2 : 1) * N, st));
    else
      PK_RET(apply_f64(P, V + (size_t)r * N, Out + (size_t)r * (P.p + 1) * N, st));
  }
  return PHIKRON_OK;
}

}  // namespace phikron
