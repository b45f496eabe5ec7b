// Float-form stage paths of polynomial degree 0, 1 (N = p + 1 = 1, 2),
// compiled apart from the other degrees so that the builds run in parallel.
#include "dg_kernels.cuh"

namespace dg {
DG_INSTANTIATE_N(template, 1, float)
DG_INSTANTIATE_N(template, 2, float)
}
