// Float-form stage paths of polynomial degree 2 (N = p + 1 = 3),
// compiled apart from the other degrees so that the builds run in parallel.
#include "dg_kernels.cuh"

namespace dg {
DG_INSTANTIATE_N(template, 3, float)
}
