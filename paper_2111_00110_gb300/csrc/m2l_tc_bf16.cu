// Tensor-core M2L, bf16 operand form: instantiation of the kernel variants.
#include "m2l_tc_kernel.cuh"

namespace fc2t2 {
FC2T2_TC_INSTANTIATE(0)
}  // namespace fc2t2
