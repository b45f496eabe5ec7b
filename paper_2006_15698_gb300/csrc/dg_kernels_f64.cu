// FP64 instantiation of the DG kernels (double state, double arithmetic).
#include "dg_kernels.cuh"

namespace dg {
template struct Launch<double>;
}
