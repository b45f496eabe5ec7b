// Float-form stage paths of polynomial degree 6 (N = p + 1 = 7),
// compiled apart from the other degrees so that the builds run in parallel.
#include "dg_kernels.cuh"

namespace dg {
DG_INSTANTIATE_N(template, 7, float)
}
