// Float-form stage paths of polynomial degree 4, 5, 6 (N = p + 1 = 5, 6, 7),
// compiled apart from the other degrees so that the builds run in parallel.
#include "dg_kernels.cuh"

namespace dg {
DG_INSTANTIATE_N(template, 5, float)
DG_INSTANTIATE_N(template, 6, float)
DG_INSTANTIATE_N(template, 7, float)
}
