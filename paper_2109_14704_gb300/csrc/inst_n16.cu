// inst_n16.cu -- kernels for N = 2^16 (words per CTA: 2^13).
#include "inst.cuh"

namespace he {
HE_DEGREE(16, 13, HE_SHAPE_FN(16, 13))
}  // namespace he

HE_DEFINE_DEGREE_OPS(16)
