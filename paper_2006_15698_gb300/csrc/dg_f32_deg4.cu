// Float-form stage paths of polynomial degree 4 (N = p + 1 = 5),
// compiled apart from the other degrees so that the builds run in parallel.
#include "dg_kernels.cuh"

namespace dg {
DG_INSTANTIATE_N(template, 5, float)
}
